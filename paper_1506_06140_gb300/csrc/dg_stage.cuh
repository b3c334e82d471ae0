// The two kernels of one RK stage (paper Sec. 2.4, eqs. dg_term2, dg_term3,
// spatial_discretisation): face fluxes, then the per-cell update.
//
// Both exploit the tensor structure of the Gauss rules: with phi_(a,b,c) =
// P~_a(x) P~_b(y) P~_c(z) (total degree a+b+c <= k), every contraction
// between modal weights and point values factorises into 1D contractions
// (sum factorisation), which cuts the multiply-adds of the direct [N x Q]
// products roughly in half at k = 2, 3.  The 1D tables travel by value in
// the kernel arguments (Tab1D), so with the loops unrolled each table entry
// is a constant-bank operand of an FMA, not a load.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "dg_internal.h"
#include "dg_physics.cuh"

namespace dgi {

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may be scheduled before the kernel ahead of it in the stream
// has finished; pdl_wait() returns once that kernel has completed and its
// writes are visible (a no-op for a kernel launched without the attribute).
// Every stage kernel calls it before its first access to global state.  No
// kernel signals its dependents early (griddepcontrol.launch_dependents): a
// dependent is released as the blocks of this grid exit.  Signalling at the
// start of every block measured slower (square advection 64^2: 0.220 against
// 0.118 ms per step), the waiting dependents' blocks holding SM slots.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// a * b + c with one rounding: the contractions below spell their
// multiply-adds out, so that a packed pair type can supply its own
__device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return fma(a, b, c); }

// Index of phi_(a,b,c) in the basis order: total degree, then a descending,
// then b descending.
template <int DIM>
__host__ __device__ constexpr int bidx(int a, int b, int c) {
  if (DIM == 2) {
    const int g = a + b;
    return g * (g + 1) / 2 + (g - a);
  }
  const int g = a + b + c;
  int pos = g * (g + 1) * (g + 2) / 6;
  for (int aa = g; aa > a; --aa) pos += g - aa + 1;
  return pos + (g - a - b);
}

// The 2D basis as seen by the sum-factorised loops: for x exponent a the y
// exponents run to lim(a) (K - a for total degree, K for the tensor product),
// and idx(a, b) is the position of phi_(a,b): by total degree, then a
// descending (the tensor product continues the order past degree K).
template <int K, int B>
struct Basis2 {
  __host__ __device__ static constexpr int lim(int a) { return B ? K : K - a; }
  __host__ __device__ static constexpr int idx(int a, int b) {
    if (B == 0 || a + b <= K) return bidx<2>(a, b, 0);
    const int m = a + b - 1 - K;  // complete degrees above K before a + b
    return (K + 1) * (K + 2) / 2 + m * K - m * (m - 1) / 2 + (K - a);
  }
};

// ---------------------------------------------------------------------------
// modal -> nodal: u(x_i, y_j[, z_k]) = sum_l w_l phi_l, factorised
template <typename real, int DIM, int K, int B = 0>
__device__ __forceinline__ void modal_to_nodal(const Tab1D<real>& T, const real* w, real* u) {
  constexpr int K1 = K + 1;
  static_assert(DIM == 2 || B == 0, "tensor-product basis: 2D");
  using BS = Basis2<K, B>;
  if constexpr (DIM == 2) {
    real t[K1][K1];  // t[a][j] = sum_b w_(a,b) P_b(y_j)
#pragma unroll
    for (int a = 0; a <= K; ++a)
#pragma unroll
      for (int j = 0; j < K1; ++j) {
        real s = real(0);
#pragma unroll
        for (int b = 0; b <= BS::lim(a); ++b) s = fmac(w[BS::idx(a, b)], T.P[b][j], s);
        t[a][j] = s;
      }
#pragma unroll
    for (int j = 0; j < K1; ++j)
#pragma unroll
      for (int i = 0; i < K1; ++i) {
        real s = real(0);
#pragma unroll
        for (int a = 0; a <= K; ++a) s = fmac(T.P[a][i], t[a][j], s);
        u[i + K1 * j] = s;
      }
  } else {
    real t1[K1][K1][K1];  // [a][b][kz] = sum_c w_(a,b,c) P_c(z_kz)
#pragma unroll
    for (int a = 0; a <= K; ++a)
#pragma unroll
      for (int b = 0; b <= K - a; ++b)
#pragma unroll
        for (int kz = 0; kz < K1; ++kz) {
          real s = real(0);
#pragma unroll
          for (int c = 0; c <= K - a - b; ++c) s = fmac(w[bidx<3>(a, b, c)], T.P[c][kz], s);
          t1[a][b][kz] = s;
        }
    real t2[K1][K1][K1];  // [a][j][kz] = sum_b t1[a][b][kz] P_b(y_j)
#pragma unroll
    for (int a = 0; a <= K; ++a)
#pragma unroll
      for (int j = 0; j < K1; ++j)
#pragma unroll
        for (int kz = 0; kz < K1; ++kz) {
          real s = real(0);
#pragma unroll
          for (int b = 0; b <= K - a; ++b) s = fmac(t1[a][b][kz], T.P[b][j], s);
          t2[a][j][kz] = s;
        }
#pragma unroll
    for (int kz = 0; kz < K1; ++kz)
#pragma unroll
      for (int j = 0; j < K1; ++j)
#pragma unroll
        for (int i = 0; i < K1; ++i) {
          real s = real(0);
#pragma unroll
          for (int a = 0; a <= K; ++a) s = fmac(T.P[a][i], t2[a][j][kz], s);
          u[i + K1 * (j + K1 * kz)] = s;
        }
  }
}

// volume integral of one variable: acc_l += sum_d sum_q f_d(q) dphi_l/dxi_d w_q
// (f_d given at the points, q = i + K1 (j + K1 k))
template <typename real, int DIM, int K, int D, int B = 0>
__device__ __forceinline__ void volume_dir(const Tab1D<real>& T, const real* f, real* acc) {
  constexpr int K1 = K + 1;
  static_assert(DIM == 2 || B == 0, "tensor-product basis: 2D");
  using BS = Basis2<K, B>;
  if constexpr (DIM == 2) {
    // derivative along axis D, weight along the other axis
#pragma unroll
    for (int e = 1; e <= K; ++e)
#pragma unroll
      for (int o = 0; o < K1; ++o) {
        real g = real(0);
#pragma unroll
        for (int i = 0; i < K1; ++i) g = fmac(f[D == 0 ? (i + K1 * o) : (o + K1 * i)], T.DW[e][i], g);
#pragma unroll
        for (int e2 = 0; e2 <= BS::lim(e); ++e2)
          acc[D == 0 ? BS::idx(e, e2) : BS::idx(e2, e)] = fmac(g, T.PW[e2][o], acc[D == 0 ? BS::idx(e, e2) : BS::idx(e2, e)]);
      }
  } else {
    // axes: D (derivative), A and BB the other two in increasing order
    constexpr int A = D == 0 ? 1 : 0;
    constexpr int BB = D == 2 ? 1 : 2;
    auto q_of = [](int d, int a, int b) {
      int x[3];
      x[D] = d;
      x[A] = a;
      x[BB] = b;
      return x[0] + K1 * (x[1] + K1 * x[2]);
    };
    auto l_of = [](int ed, int ea, int eb) {
      int e[3];
      e[D] = ed;
      e[A] = ea;
      e[BB] = eb;
      return bidx<3>(e[0], e[1], e[2]);
    };
#pragma unroll
    for (int ed = 1; ed <= K; ++ed) {
      real g1[K1][K1];  // [ia][ib] = sum_id f DW[ed][id]
#pragma unroll
      for (int ia = 0; ia < K1; ++ia)
#pragma unroll
        for (int ib = 0; ib < K1; ++ib) {
          real s = real(0);
#pragma unroll
          for (int id = 0; id < K1; ++id) s = fmac(f[q_of(id, ia, ib)], T.DW[ed][id], s);
          g1[ia][ib] = s;
        }
#pragma unroll
      for (int ea = 0; ea <= K - ed; ++ea)
#pragma unroll
        for (int ib = 0; ib < K1; ++ib) {
          real g2 = real(0);
#pragma unroll
          for (int ia = 0; ia < K1; ++ia) g2 = fmac(g1[ia][ib], T.PW[ea][ia], g2);
#pragma unroll
          for (int eb = 0; eb <= K - ed - ea; ++eb) acc[l_of(ed, ea, eb)] = fmac(g2, T.PW[eb][ib], acc[l_of(ed, ea, eb)]);
        }
    }
  }
}

// projection of a field given at the volume points onto the basis:
// acc_l += h * sum_q s_q phi_l(xi_q) w_q (q = i + K1 (j + K1 k)), sum-factorised
// with the weighted 1D tables along every axis
template <typename real, int DIM, int K, int B = 0>
__device__ __forceinline__ void source_project(const Tab1D<real>& T, const real* s, real h, real* acc) {
  constexpr int K1 = K + 1;
  static_assert(DIM == 2 || B == 0, "tensor-product basis: 2D");
  using BS = Basis2<K, B>;
  if constexpr (DIM == 2) {
#pragma unroll
    for (int e1 = 0; e1 <= K; ++e1) {
      real g[K1];
#pragma unroll
      for (int i2 = 0; i2 < K1; ++i2) {
        real t = real(0);
#pragma unroll
        for (int i1 = 0; i1 < K1; ++i1) t = fmac(s[i1 + K1 * i2], T.PW[e1][i1], t);
        g[i2] = t;
      }
#pragma unroll
      for (int e2 = 0; e2 <= BS::lim(e1); ++e2) {
        real t = real(0);
#pragma unroll
        for (int i2 = 0; i2 < K1; ++i2) t = fmac(g[i2], T.PW[e2][i2], t);
        acc[BS::idx(e1, e2)] = fmac(h, t, acc[BS::idx(e1, e2)]);
      }
    }
  } else {
#pragma unroll
    for (int e1 = 0; e1 <= K; ++e1) {
      real g1[K1][K1];
#pragma unroll
      for (int i2 = 0; i2 < K1; ++i2)
#pragma unroll
        for (int i3 = 0; i3 < K1; ++i3) {
          real t = real(0);
#pragma unroll
          for (int i1 = 0; i1 < K1; ++i1) t = fmac(s[i1 + K1 * (i2 + K1 * i3)], T.PW[e1][i1], t);
          g1[i2][i3] = t;
        }
#pragma unroll
      for (int e2 = 0; e2 <= K - e1; ++e2) {
        real g2[K1];
#pragma unroll
        for (int i3 = 0; i3 < K1; ++i3) {
          real t = real(0);
#pragma unroll
          for (int i2 = 0; i2 < K1; ++i2) t = fmac(g1[i2][i3], T.PW[e2][i2], t);
          g2[i3] = t;
        }
#pragma unroll
        for (int e3 = 0; e3 <= K - e1 - e2; ++e3) {
          real t = real(0);
#pragma unroll
          for (int i3 = 0; i3 < K1; ++i3) t = fmac(g2[i3], T.PW[e3][i3], t);
          acc[bidx<3>(e1, e2, e3)] = fmac(h, t, acc[bidx<3>(e1, e2, e3)]);
        }
      }
    }
  }
}

// surface integral of one variable over side (DIR, S) of the cell:
// acc_l -= sg * sum_q fbar_q phi_l(face point q) w_q, with the face's points
// given by the weighted tables PW0 (and PW1): PW[e][q] = P_e(x_q) w_q at the
// Gauss nodes (T.PW), or at a half of them for sub-faces (T.PWH[h]).
template <typename real, int DIM, int K, int DIR, int S, int B = 0>
__device__ __forceinline__ void surface_side(const Tab1D<real>& T, const real (&PW0)[4][4],
                                             const real (&PW1)[4][4], const real* fq, real scale,
                                             real* acc) {
  constexpr int K1 = K + 1;
  static_assert(DIM == 2 || B == 0, "tensor-product basis: 2D");
  using BS = Basis2<K, B>;
  const real ssg = S ? -scale : scale;  // times minus the outward normal's sign
  if constexpr (DIM == 2) {
    constexpr int TA = DIR == 0 ? 1 : 0;
    real G[K1];
#pragma unroll
    for (int e = 0; e <= K; ++e) {
      real s = real(0);
#pragma unroll
      for (int q = 0; q < K1; ++q) s = fmac(fq[q], PW0[e][q], s);
      G[e] = s * ssg;
    }
#pragma unroll
    for (int ed = 0; ed <= K; ++ed)
#pragma unroll
      for (int et = 0; et <= BS::lim(ed); ++et)
        acc[TA == 1 ? BS::idx(ed, et) : BS::idx(et, ed)] = fmac(T.PE[S][ed], G[et], acc[TA == 1 ? BS::idx(ed, et) : BS::idx(et, ed)]);
  } else {
    constexpr int A = DIR == 0 ? 1 : 0;  // tangential axes, increasing
    constexpr int BB = DIR == 2 ? 1 : 2;
    real H[K1][K1];  // [ea][qb] = sum_qa f w P_ea
#pragma unroll
    for (int ea = 0; ea <= K; ++ea)
#pragma unroll
      for (int qb = 0; qb < K1; ++qb) {
        real s = real(0);
#pragma unroll
        for (int qa = 0; qa < K1; ++qa) s = fmac(fq[qa + K1 * qb], PW0[ea][qa], s);
        H[ea][qb] = s;
      }
#pragma unroll
    for (int ea = 0; ea <= K; ++ea)
#pragma unroll
      for (int eb = 0; eb <= K - ea; ++eb) {
        real s = real(0);
#pragma unroll
        for (int qb = 0; qb < K1; ++qb) s = fmac(H[ea][qb], PW1[eb][qb], s);
        s *= ssg;
#pragma unroll
        for (int ed = 0; ed <= K - ea - eb; ++ed) {
          int e[3];
          e[DIR] = ed;
          e[A] = ea;
          e[BB] = eb;
          acc[bidx<3>(e[0], e[1], e[2])] = fmac(T.PE[S][ed], s, acc[bidx<3>(e[0], e[1], e[2])]);
        }
      }
  }
}

// 3D faces: the face-flux array holds, per variable, the moments
//   M(ea, eb) = sum_q f(q) P~_ea(x_qa) P~_eb(x_qb) w_qa w_qb,  ea + eb <= k,
// of the flux at the face's Gauss points (q = qa + (k+1) qb along the two
// tangential axes in increasing order): the sum-factorised first two
// contractions of surface_side, done once per face instead of once per side.
template <int K>
__host__ __device__ constexpr int face_moment(int ea, int eb) {
  return ea * (K + 1) - ea * (ea - 1) / 2 + eb;
}

template <typename real, int K>
__device__ __forceinline__ void face_moments(const Tab1D<real>& T, const real* fq, real* M) {
  constexpr int K1 = K + 1;
  real H[K1][K1];  // [ea][qb] = sum_qa f w P_ea
#pragma unroll
  for (int ea = 0; ea <= K; ++ea)
#pragma unroll
    for (int qb = 0; qb < K1; ++qb) {
      real s = real(0);
#pragma unroll
      for (int qa = 0; qa < K1; ++qa) s = fmac(fq[qa + K1 * qb], T.PW[ea][qa], s);
      H[ea][qb] = s;
    }
#pragma unroll
  for (int ea = 0; ea <= K; ++ea)
#pragma unroll
    for (int eb = 0; eb <= K - ea; ++eb) {
      real s = real(0);
#pragma unroll
      for (int qb = 0; qb < K1; ++qb) s = fmac(H[ea][qb], T.PW[eb][qb], s);
      M[face_moment<K>(ea, eb)] = s;
    }
}

// acc_l -= sg * scale * sum over the face of f phi_l, from the face moments:
// phi_(ed, ea, eb) restricted to side (DIR, S) is P~_ed(+-1) P~_ea P~_eb
template <typename real, int K, int DIR, int S>
__device__ __forceinline__ void surface_side_moments(const Tab1D<real>& T, const real* M, real scale, real* acc) {
  constexpr int A = DIR == 0 ? 1 : 0;  // tangential axes, increasing
  constexpr int BB = DIR == 2 ? 1 : 2;
  const real ssg = S ? -scale : scale;
#pragma unroll
  for (int ea = 0; ea <= K; ++ea)
#pragma unroll
    for (int eb = 0; eb <= K - ea; ++eb) {
      const real s = M[face_moment<K>(ea, eb)] * ssg;
#pragma unroll
      for (int ed = 0; ed <= K - ea - eb; ++ed) {
        int e[3];
        e[DIR] = ed;
        e[A] = ea;
        e[BB] = eb;
        acc[bidx<3>(e[0], e[1], e[2])] = fmac(T.PE[S][ed], s, acc[bidx<3>(e[0], e[1], e[2])]);
      }
    }
}

// the moments of a sub-face (quadrant h of the coarse face, in the sub-face's
// own coordinates) as moments against the coarse face's Legendre products:
// P~_a on a half interval is sum_{b <= a} TH[half][a][b] P~_b of the half's
// own coordinate, exactly
template <typename real, int K>
__device__ __forceinline__ void sub_to_coarse_moments(const Tab1D<real>& T, int h, const real* Ms, real* Mc) {
  constexpr int K1 = K + 1;
  const int h0 = h & 1, h1 = (h >> 1) & 1;
  real G[K1][K1];  // [ea'][eb] = sum_{eb' <= eb} TH[h1][eb][eb'] Ms(ea', eb'), ea' + eb <= K
#pragma unroll
  for (int ea = 0; ea <= K; ++ea)
#pragma unroll
    for (int eb = 0; eb <= K - ea; ++eb) {
      real s = real(0);
#pragma unroll
      for (int eb2 = 0; eb2 <= eb; ++eb2) s = fmac(T.TH[h1][eb][eb2], Ms[face_moment<K>(ea, eb2)], s);
      G[ea][eb] = s;
    }
#pragma unroll
  for (int ea = 0; ea <= K; ++ea)
#pragma unroll
    for (int eb = 0; eb <= K - ea; ++eb) {
      real s = real(0);
#pragma unroll
      for (int ea2 = 0; ea2 <= ea; ++ea2) s = fmac(T.TH[h0][ea][ea2], G[ea2][eb], s);
      Mc[face_moment<K>(ea, eb)] = s;
    }
}

// Whether the face-flux array holds face moments: always in 3D, and in 2D
// for an FP64 state (2D: M(e) = sum_q f(q) P~_e(x_q) w_q, e <= k, as many as
// points; the FP32 2D kernels -- tensor-core, one thread per cell, packed
// pairs -- read point values).
template <typename real, int DIM>
struct FaceMoments {
  static constexpr bool ON = DIM == 3 || std::is_same<real, double>::value;
};

template <typename real, int K>
__device__ __forceinline__ void face_moments_2d(const Tab1D<real>& T, const real* fq, real* M) {
#pragma unroll
  for (int e = 0; e <= K; ++e) {
    real s = real(0);
#pragma unroll
    for (int q = 0; q <= K; ++q) s = fmac(fq[q], T.PW[e][q], s);
    M[e] = s;
  }
}

// the second half of surface_side (2D) from the face moments
template <typename real, int K, int DIR, int S, int B = 0>
__device__ __forceinline__ void surface_side_moments_2d(const Tab1D<real>& T, const real* M, real scale, real* acc) {
  using BS = Basis2<K, B>;
  constexpr int TA = DIR == 0 ? 1 : 0;
  const real ssg = S ? -scale : scale;
  real G[K + 1];
#pragma unroll
  for (int e = 0; e <= K; ++e) G[e] = M[e] * ssg;
#pragma unroll
  for (int ed = 0; ed <= K; ++ed)
#pragma unroll
    for (int et = 0; et <= BS::lim(ed); ++et)
      acc[TA == 1 ? BS::idx(ed, et) : BS::idx(et, ed)] = fmac(T.PE[S][ed], G[et], acc[TA == 1 ? BS::idx(ed, et) : BS::idx(et, ed)]);
}

// sub-face moments (half h of the coarse face, own coordinate) as moments
// against the coarse face's Legendre polynomials
template <typename real, int K>
__device__ __forceinline__ void sub_to_coarse_moments_2d(const Tab1D<real>& T, int h, const real* Ms, real* Mc) {
#pragma unroll
  for (int e = 0; e <= K; ++e) {
    real s = real(0);
#pragma unroll
    for (int e2 = 0; e2 <= e; ++e2) s = fmac(T.TH[h][e][e2], Ms[e2], s);
    Mc[e] = s;
  }
}

// trace of one variable on side (DIR, S) at the face points given by PT0/PT1
template <typename real, int DIM, int K, int DIR, int B = 0>
__device__ __forceinline__ void face_trace(const Tab1D<real>& T, const real* w, int s,
                                           const real (&PT0)[4][4], const real (&PT1)[4][4],
                                           real* u) {
  constexpr int K1 = K + 1;
  static_assert(DIM == 2 || B == 0, "tensor-product basis: 2D");
  using BS = Basis2<K, B>;
  if constexpr (DIM == 2) {
    real t[K1];
#pragma unroll
    for (int et = 0; et <= K; ++et) {
      real acc = real(0);
#pragma unroll
      for (int ed = 0; ed <= BS::lim(et); ++ed)
        acc = fmac(w[DIR == 0 ? BS::idx(ed, et) : BS::idx(et, ed)], T.PE[s][ed], acc);
      t[et] = acc;
    }
#pragma unroll
    for (int q = 0; q < K1; ++q) {
      real acc = real(0);
#pragma unroll
      for (int et = 0; et <= K; ++et) acc = fmac(t[et], PT0[et][q], acc);
      u[q] = acc;
    }
  } else {
    constexpr int A = DIR == 0 ? 1 : 0;
    constexpr int BB = DIR == 2 ? 1 : 2;
    real t[K1][K1];
#pragma unroll
    for (int ea = 0; ea <= K; ++ea)
#pragma unroll
      for (int eb = 0; eb <= K - ea; ++eb) {
        real acc = real(0);
#pragma unroll
        for (int ed = 0; ed <= K - ea - eb; ++ed) {
          int e[3];
          e[DIR] = ed;
          e[A] = ea;
          e[BB] = eb;
          acc = fmac(w[bidx<3>(e[0], e[1], e[2])], T.PE[s][ed], acc);
        }
        t[ea][eb] = acc;
      }
#pragma unroll
    for (int ea = 0; ea <= K; ++ea) {
      real h[K1];
#pragma unroll
      for (int qb = 0; qb < K1; ++qb) {
        real acc = real(0);
#pragma unroll
        for (int eb = 0; eb <= K - ea; ++eb) acc = fmac(t[ea][eb], PT1[eb][qb], acc);
        h[qb] = acc;
      }
#pragma unroll
      for (int qb = 0; qb < K1; ++qb)
#pragma unroll
        for (int qa = 0; qa < K1; ++qa) {
          if (ea == 0) u[qa + K1 * qb] = real(0);
          u[qa + K1 * qb] = fmac(PT0[ea][qa], h[qb], u[qa + K1 * qb]);
        }
    }
  }
}

// ===========================================================================
// Face kernel: FB faces per block, NV threads per face.
//   1. thread (face, var): load both cells' weights of its variable and
//      compute the traces at all face points -> shared memory;
//   2. thread (face, point): HLLC flux -> F[var][point][face] (coalesced);
//      in 3D into shared memory, and then
//   3. (3D) thread (face, var): the face moments of the flux -> F[var][moment][face].
// A variant > 0 marks the coarse side of a hanging face: its points are a
// half (2D) or quarter (3D) of the cell face.

// Faces per block: FB (default 32) is a template parameter; instantiated for
// 16, 32 and 64, selected at launch (StageArgs::face_tile).
template <typename real, int DIM, int K>
struct FaceTile {
  using S = Shape<DIM, K>;
  static constexpr int FB = 32;
  static constexpr int FB_MAX = 64;
  static constexpr size_t smem(int fb) { return (size_t)2 * S::NV * S::QF * fb * sizeof(real); }
};

template <typename real, int DIM, int K, int DIR, int B = 0>
__device__ __forceinline__ void trace_side(const StageArgs<real>& a, int cell, int s, int var,
                                           int v, real* u) {
  using S = Shape<DIM, K, B>;
  const Tab1D<real>& T = a.t1;
  const int nc = a.m.ncells;
  real w[S::N];
#pragma unroll
  for (int l = 0; l < S::N; ++l) w[l] = a.U[(size_t)(v * S::N + l) * nc + cell];
  if (var == 0) {
    face_trace<real, DIM, K, DIR, B>(T, w, s, T.P, T.P, u);
  } else {
    const int h0 = (var - 1) & 1, h1 = ((var - 1) >> 1) & 1;
    face_trace<real, DIM, K, DIR, B>(T, w, s, T.PH[h0], T.PH[h1], u);
  }
}

// the work of one block (faces bid*FB ..) with FB*NV threads; the kernel
// below and the persistent step kernel run it
template <typename real, int DIM, int K, int FB, int B = 0>
__device__ __forceinline__ void face_flux_body(const StageArgs<real>& a, int bid) {
  using S = Shape<DIM, K, B>;
  constexpr int THREADS = FB * S::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sT = reinterpret_cast<real*>(smem_raw);  // [2 sides][NV][QF][FB]
  const int nf = a.m.nfaces;
  const int fl = threadIdx.x % FB, v = threadIdx.x / FB;
  const int f = bid * FB + fl;
  int dir = 0;
  if (f < nf) {
    const unsigned info = a.m.finfo[f];
    dir = info & 3;
    const int vm = (info >> 2) & 7, vp = (info >> 5) & 7;
    const int cm = a.m.fm[f], cp = a.m.fp[f];
    real um[S::QF], up[S::QF];
    // the minus cell sees the face as its + side (s = 1), the plus cell as its - side
    auto trace = [&](int cell, int s, int var, real* u) {
      if (dir == 0) trace_side<real, DIM, K, 0, B>(a, cell, s, var, v, u);
      else if (dir == 1) trace_side<real, DIM, K, 1, B>(a, cell, s, var, v, u);
      else if constexpr (DIM == 3) trace_side<real, DIM, K, DIM - 1, B>(a, cell, s, var, v, u);
    };
    if (cm >= 0) trace(cm, 1, vm, um);
    if (cp >= 0) trace(cp, 0, vp, up);
    if (cm < 0) {
#pragma unroll
      for (int q = 0; q < S::QF; ++q) um[q] = up[q];
    }
    if (cp < 0) {
#pragma unroll
      for (int q = 0; q < S::QF; ++q) up[q] = um[q];
    }
#pragma unroll
    for (int q = 0; q < S::QF; ++q) {
      sT[((0 * S::NV + v) * S::QF + q) * FB + fl] = um[q];
      sT[((1 * S::NV + v) * S::QF + q) * FB + fl] = up[q];
    }
  }
  __syncthreads();
  // HLLC at every (face, point) of the block
  const real gamma = a.gam;
  for (int item = threadIdx.x; item < FB * S::QF; item += THREADS) {
    const int ff = item % FB, q = item / FB;
    const int f2 = bid * FB + ff;
    if (f2 >= nf) continue;
    const int d2 = a.m.finfo[f2] & 3;
    real uL[S::NV], uR[S::NV], Fl[S::NV];
#pragma unroll
    for (int vv = 0; vv < S::NV; ++vv) {
      uL[vv] = sT[((0 * S::NV + vv) * S::QF + q) * FB + ff];
      uR[vv] = sT[((1 * S::NV + vv) * S::QF + q) * FB + ff];
    }
    if (d2 == 0) hllc_flux<real, DIM>(uL, uR, 0, gamma, Fl);
    else if (d2 == 1) hllc_flux<real, DIM>(uL, uR, 1, gamma, Fl);
    else hllc_flux<real, DIM>(uL, uR, DIM - 1, gamma, Fl);
    if constexpr (FaceMoments<real, DIM>::ON) {
      // over the minus trace of this point, which only this item reads
#pragma unroll
      for (int vv = 0; vv < S::NV; ++vv) sT[((0 * S::NV + vv) * S::QF + q) * FB + ff] = Fl[vv];
    } else {
#pragma unroll
      for (int vv = 0; vv < S::NV; ++vv) a.F[((size_t)vv * S::QF + q) * nf + f2] = Fl[vv];
    }
  }
  if constexpr (FaceMoments<real, DIM>::ON) {
    // thread (face, variable): the face moments of its variable's flux
    __syncthreads();
    if (f < nf) {
      real fq[S::QF], M[S::FV];
#pragma unroll
      for (int q = 0; q < S::QF; ++q) fq[q] = sT[((0 * S::NV + v) * S::QF + q) * FB + fl];
      if constexpr (DIM == 3) face_moments<real, K>(a.t1, fq, M);
      else face_moments_2d<real, K>(a.t1, fq, M);
#pragma unroll
      for (int m = 0; m < S::FV; ++m) a.F[((size_t)v * S::FV + m) * nf + f] = M[m];
    }
  }
  (void)dir;
}

template <typename real, int DIM, int K, int FB, int B = 0>
__global__ void __launch_bounds__(FB * Shape<DIM, K>::NV)
    face_flux_kernel(const StageArgs<real> a) {
  pdl_wait();
  face_flux_body<real, DIM, K, FB, B>(a, blockIdx.x);
}

// ===========================================================================
// Cell kernel: TC cells per block, NV threads per cell (thread <-> variable).
//   1. thread (cell, var): its variable's weights -> nodal values at the
//      (k+1)^d Gauss points (sum factorisation) -> shared memory;
//   2. thread (cell, p): Euler fluxes at points p, p+NV, ... -> shared memory;
//   3. thread (cell, var): volume integral (sum factorisation) minus the
//      surface integral of the stored face fluxes, times 2^(1-d)/dx;
//   4. epilogue: out_o = sum_r C[o][r] in_r + ck[o] dt dW/dt.

template <typename real, int DIM, int K>
struct CellTile {
  using S = Shape<DIM, K>;
  // per cell: the nodal state [NV][Q] and the point fluxes [DIM][NV][Q].  The
  // fluxes of direction 0 overwrite the nodal state (a thread overwrites only
  // the point values it has itself just read), except in the gravity variant,
  // whose source term reads the nodal state after the fluxes.
  static constexpr size_t PER_CELL = (size_t)(S::NV * S::Q + DIM * S::NV * S::Q) * sizeof(real);
  static constexpr size_t PER_CELL_ALIASED = (size_t)(DIM * S::NV * S::Q) * sizeof(real);
  // cells per block: TC (the default) is a template parameter, instantiated
  // for 16, 32 and 64 up to TC_MAX and selected at launch (StageArgs::cell_tile)
  static constexpr int TC = PER_CELL * 32 > 96 * 1024 ? 16 : 32;
  static constexpr int TC_MAX = PER_CELL * 64 <= 200 * 1024 ? 64 : (PER_CELL * 32 <= 200 * 1024 ? 32 : 16);
  static constexpr size_t smem(int tc, bool grav = false) { return (grav ? PER_CELL : PER_CELL_ALIASED) * tc; }
  // register targets of the FP32 kernels (latency- or issue-bound): 3D asks
  // for 20 resident warps per SM (at most ~102 registers per thread), 2D for
  // 48 registers per thread up to k = 2 and 64 at k = 3; FP64 (FP64-pipe
  // bound) has none
  static constexpr int fit(int tc, int regs) { return 65536 / (tc * S::NV * regs); }
  static constexpr int min_blocks(int tc) {
    return sizeof(real) != 4 ? 1
           : DIM == 3        ? (640 / (tc * S::NV) > 1 ? 640 / (tc * S::NV) : 1)
                             : (fit(tc, K <= 2 ? 48 : 64) > 1 ? fit(tc, K <= 2 ? 48 : 64) : 1);
  }
};

// Face fluxes of the conforming sides of a cell are loaded at the start of
// the cell kernel (when they fit in 64 registers) so that their latency
// overlaps the volume phase; a coarse side's sub-face fluxes load on use.
template <typename real, int DIM, int K>
struct FacePrefetch {
  static constexpr bool ON = 2 * DIM * Shape<DIM, K>::FV * sizeof(real) <= 256;
};

template <typename real, int DIM, int K>
__device__ __forceinline__ void prefetch_faces(const StageArgs<real>& a, int c, int v, unsigned coarse,
                                               real (&fp)[2 * DIM][Shape<DIM, K>::FV]) {
  using S = Shape<DIM, K>;
  const int nc = a.m.ncells, nf = a.m.nfaces;
#pragma unroll
  for (int sd = 0; sd < 2 * DIM; ++sd) {
    const bool conf = !((coarse >> sd) & 1);
    const int e0 = conf ? a.m.sface[(size_t)sd * nc + c] : 0;
#pragma unroll
    for (int q = 0; q < S::FV; ++q) fp[sd][q] = conf ? a.F[((size_t)v * S::FV + q) * nf + e0] : real(0);
  }
}

template <typename real, int DIM, int K, int SD, int B = 0>
__device__ __forceinline__ void surface_from_faces(const StageArgs<real>& a, int c, int v,
                                                   unsigned coarse, const real* fpre, real* acc) {
  using S = Shape<DIM, K>;
  constexpr int DIR = SD >> 1, SS = SD & 1;
  const Tab1D<real>& T = a.t1;
  const int nc = a.m.ncells, nf = a.m.nfaces;
  real fq[S::FV];
  if (!((coarse >> SD) & 1)) {
    if (fpre) {
#pragma unroll
      for (int q = 0; q < S::FV; ++q) fq[q] = fpre[q];
    } else {
      const int e0 = a.m.sface[(size_t)SD * nc + c];
#pragma unroll
      for (int q = 0; q < S::FV; ++q) fq[q] = a.F[((size_t)v * S::FV + q) * nf + e0];
    }
    if constexpr (DIM == 3) surface_side_moments<real, K, DIR, SS>(T, fq, real(1), acc);
    else if constexpr (FaceMoments<real, DIM>::ON) surface_side_moments_2d<real, K, DIR, SS, B>(T, fq, real(1), acc);
    else surface_side<real, DIM, K, DIR, SS, B>(T, T.PW, T.PW, fq, real(1), acc);
  } else {
    const int e0 = a.m.sface[(size_t)SD * nc + c];
    // coarse side of a hanging face: NSUB sub-faces in quadrant order
    const real sub = real(1) / real(S::NSUB);
#pragma unroll
    for (int h = 0; h < S::NSUB; ++h) {
#pragma unroll
      for (int q = 0; q < S::FV; ++q) fq[q] = a.F[((size_t)v * S::FV + q) * nf + e0 + h];
      if constexpr (DIM == 3) {
        real Mc[S::NM];
        sub_to_coarse_moments<real, K>(T, h, fq, Mc);
        surface_side_moments<real, K, DIR, SS>(T, Mc, sub, acc);
      } else if constexpr (FaceMoments<real, DIM>::ON) {
        real Mc[S::FV];
        sub_to_coarse_moments_2d<real, K>(T, h, fq, Mc);
        surface_side_moments_2d<real, K, DIR, SS, B>(T, Mc, sub, acc);
      } else {
        surface_side<real, DIM, K, DIR, SS, B>(T, T.PWH[h & 1], T.PWH[(h >> 1) & 1], fq, sub, acc);
      }
    }
  }
}

// out_o = ck_o sc acc + sum_r C[o][r] in_r for the weights of variable v of
// cell c (sc = dt * 2^(1-d)/dx), the terms added in that order; the
// stage-program loops run outside the coefficient loop, so each coefficient
// costs one load and one FMA per input; w: the cell's weights of U
template <typename real, int N>
__device__ __forceinline__ void stage_epilogue(const StageArgs<real>& a, int c, int v, real sc, const real* acc,
                                               const real* w) {
  const int nc = a.m.ncells;
  const size_t i0 = (size_t)(v * N) * nc + c;
#pragma unroll
  for (int oo = 0; oo < MAX_OUT; ++oo) {
    if (oo >= a.n_out) break;
    const real ckv = a.ck[oo] * sc;
    real val[N];
#pragma unroll
    for (int j = 0; j < N; ++j) val[j] = ckv * acc[j];
#pragma unroll
    for (int r = 0; r < MAX_IN; ++r) {
      if (r >= a.n_in) break;
      const real cr = a.C[oo][r];
      if (cr == real(0)) continue;
      const real* src = a.in[r];
      if (src == a.U) {
#pragma unroll
        for (int j = 0; j < N; ++j) val[j] += cr * w[j];
      } else {
#pragma unroll
        for (int j = 0; j < N; ++j) val[j] += cr * src[i0 + (size_t)j * nc];
      }
    }
    real* dst = a.out[oo];
#pragma unroll
    for (int j = 0; j < N; ++j) dst[i0 + (size_t)j * nc] = val[j];
  }
}

// the work of one block (cells bid*TC ..) with TC*NV threads; the kernel
// below and the persistent step kernel run it
template <typename real, int DIM, int K, int TC, bool GRAV = false, int B = 0>
__device__ __forceinline__ void cell_update_body(const StageArgs<real>& a, int bid) {
  using S = Shape<DIM, K, B>;
  constexpr int NV = S::NV, Q = S::Q, N = S::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sU = reinterpret_cast<real*>(smem_raw);    // [NV][Q][TC]
  real* sF = GRAV ? sU + NV * Q * TC : sU;         // [DIM][NV][Q][TC] (direction 0 over sU)
  const int tc = threadIdx.x % TC, v = threadIdx.x / TC;
  const int nc = a.m.ncells;
  const int c = bid * TC + tc;
  const bool valid = c < nc;
  const Tab1D<real>& T = a.t1;
  constexpr bool PF = FacePrefetch<real, DIM, K>::ON;
  const unsigned coarse = valid ? a.m.scoarse[c] : 0u;
  real fpre[PF ? 2 * DIM : 1][S::FV];
  if constexpr (PF) {
    if (valid) prefetch_faces<real, DIM, K>(a, c, v, coarse, fpre);
  }

  // 1. weights of this variable -> nodal values
  real w[N];
#pragma unroll
  for (int l = 0; l < N; ++l)
    w[l] = valid ? a.U[(size_t)(v * N + l) * nc + c] : ((v == 0 && l == 0) ? real(1) : real(0));
  {
    real u[Q];
    modal_to_nodal<real, DIM, K, B>(T, w, u);
#pragma unroll
    for (int q = 0; q < Q; ++q) sU[(v * Q + q) * TC + tc] = u[q];
  }
  __syncthreads();

  // 2. Euler fluxes at the points of this thread
  const real g1 = a.gm1;
  for (int q = v; q < Q; q += NV) {
    real u[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) u[vv] = sU[(vv * Q + q) * TC + tc];
    real f[DIM][NV];
    euler_flux_all<real, DIM>(u, g1, f);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) sF[((d * NV + vv) * Q + q) * TC + tc] = f[d][vv];
  }
  __syncthreads();
  if (!valid) return;

  // 3. volume and surface integrals of this variable
  real acc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l] = real(0);
  {
    real f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = sF[((0 * NV + v) * Q + q) * TC + tc];
    volume_dir<real, DIM, K, 0, B>(T, f, acc);
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = sF[((1 * NV + v) * Q + q) * TC + tc];
    volume_dir<real, DIM, K, 1, B>(T, f, acc);
    if constexpr (DIM == 3) {
#pragma unroll
      for (int q = 0; q < Q; ++q) f[q] = sF[((2 * NV + v) * Q + q) * TC + tc];
      volume_dir<real, DIM, K, DIM - 1, B>(T, f, acc);
    }
  }
  surface_from_faces<real, DIM, K, 0, B>(a, c, v, coarse, PF ? fpre[0] : nullptr, acc);
  surface_from_faces<real, DIM, K, 1, B>(a, c, v, coarse, PF ? fpre[1] : nullptr, acc);
  surface_from_faces<real, DIM, K, 2, B>(a, c, v, coarse, PF ? fpre[2 % (PF ? 2 * DIM : 1)] : nullptr, acc);
  surface_from_faces<real, DIM, K, 3, B>(a, c, v, coarse, PF ? fpre[3 % (PF ? 2 * DIM : 1)] : nullptr, acc);
  if constexpr (DIM == 3) {
    surface_from_faces<real, DIM, K, 4, B>(a, c, v, coarse, PF ? fpre[4 % (PF ? 2 * DIM : 1)] : nullptr, acc);
    surface_from_faces<real, DIM, K, 5, B>(a, c, v, coarse, PF ? fpre[5 % (PF ? 2 * DIM : 1)] : nullptr, acc);
  }

  // 4. epilogue
  const int pb = cell_problem(a.m, c);
  const real pre = a.pre_prob ? a.pre_prob[pb] : a.pre[a.m.level[c]];
  if constexpr (GRAV) {
    // gravity source (eq. gravity_term): s = (0, rho a, m . a) at the volume
    // points; pre * (dx/2) * sum_q s_q phi_j w_q = 2^-d sum_q s_q phi_j w_q
    if (v > 0) {
      real sq[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (v <= DIM) {
          sq[q] = sU[(0 * Q + q) * TC + tc] * a.accel[((size_t)(v - 1) * Q + q) * nc + c];
        } else {
          real t = real(0);
#pragma unroll
          for (int d = 0; d < DIM; ++d) t += sU[((1 + d) * Q + q) * TC + tc] * a.accel[((size_t)d * Q + q) * nc + c];
          sq[q] = t;
        }
      }
      source_project<real, DIM, K, B>(T, sq, real(1) / (real(1 << DIM) * pre), acc);
    }
  }
  stage_epilogue<real, N>(a, c, v, pre * (a.dt ? real(a.dt[pb]) : real(1)), acc, w);
}

template <typename real, int DIM, int K, int TC, bool GRAV = false, int B = 0>
__global__ void __launch_bounds__(TC * Shape<DIM, K>::NV, CellTile<real, DIM, K>::min_blocks(TC))
    cell_update_kernel(const StageArgs<real> a) {
  pdl_wait();
  cell_update_body<real, DIM, K, TC, GRAV, B>(a, blockIdx.x);
}

}  // namespace dgi
