// Cell kernel of a 2D FP32 stage with two variables per thread, as packed
// FP32 pairs (Blackwell's paired FP32 multiply-add: two lanes per
// instruction, each rounded as a scalar fmaf).  Thread (cell, p) carries the
// variables 2p and 2p+1 through the same sum-factorised contractions as the
// one-variable-per-thread cell kernel -- modal -> nodal, volume and surface
// integrals (Sec. 2.4, eqs. dg_term1-3) -- with every table entry duplicated
// into both lanes, so each multiply-add serves two variables.  Per lane the
// operations and their order are those of the scalar kernel, so the results
// are the same bits.
#pragma once
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_physics.cuh"
#include "dg_stage.cuh"

namespace dgi {

struct alignas(8) f32x2 {
  float2 v;
  f32x2() = default;
  __host__ __device__ f32x2(float a) { v.x = a; v.y = a; }
  __host__ __device__ f32x2(float a, float b) { v.x = a; v.y = b; }
};

__device__ __forceinline__ f32x2 fmac(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  r.v = __ffma2_rn(a.v, b.v, c.v);
  return r;
}
__device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) {
  f32x2 r;
  r.v = __fmul2_rn(a.v, b.v);
  return r;
}
__device__ __forceinline__ f32x2 operator-(f32x2 a) { return f32x2(-a.v.x, -a.v.y); }

// stage arguments plus the 1D tables with every entry in both lanes
struct X2Args {
  StageArgs<float> a;
  Tab1D<f32x2> t2;
};

template <int K, int TC>
struct X2Tile {
  using S = Shape<2, K>;
  static constexpr int NP = S::NV / 2;  // variable pairs
  static constexpr int THREADS = TC * NP;
  // point fluxes [2 directions][NP][Q][TC] pairs; direction 0 over the nodal values
  static constexpr size_t SMEM = (size_t)2 * NP * S::Q * TC * sizeof(f32x2);
};

template <int K, int TC>
__global__ void __launch_bounds__(X2Tile<K, TC>::THREADS, TC == 64 ? 4 : 8)
    cell_update_x2_kernel(const X2Args x) {
  using S = Shape<2, K>;
  using XT = X2Tile<K, TC>;
  constexpr int NV = S::NV, NP = XT::NP, N = S::N, Q = S::Q, QF = S::QF;
  const StageArgs<float>& a = x.a;
  const Tab1D<f32x2>& T = x.t2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  f32x2* sU = reinterpret_cast<f32x2*>(smem_raw);  // [NP][Q][TC]
  f32x2* sF = sU;                                  // [2][NP][Q][TC], direction 0 over sU
  const int tc = threadIdx.x % TC, p = threadIdx.x / TC;
  const int nc = a.m.ncells, nf = a.m.nfaces;
  const int c = blockIdx.x * TC + tc;
  const bool valid = c < nc;
  const int v0 = 2 * p, v1 = 2 * p + 1;
  const unsigned coarse = valid ? a.m.scoarse[c] : 0u;

  // 1. weights of the pair -> nodal values (a padding cell: the unit density state)
  f32x2 w[N];
#pragma unroll
  for (int l = 0; l < N; ++l)
    w[l] = valid ? f32x2(a.U[(size_t)(v0 * N + l) * nc + c], a.U[(size_t)(v1 * N + l) * nc + c])
                 : f32x2((p == 0 && l == 0) ? 1.0f : 0.0f, 0.0f);
  {
    f32x2 u[Q];
    modal_to_nodal<f32x2, 2, K>(T, w, u);
#pragma unroll
    for (int q = 0; q < Q; ++q) sU[(p * Q + q) * TC + tc] = u[q];
  }
  __syncthreads();

  // 2. Euler fluxes at the points of this thread (all variables of a point)
  const float g1 = a.gm1;
  for (int q = p; q < Q; q += NP) {
    float u[NV];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      const f32x2 t = sU[(pp * Q + q) * TC + tc];
      u[2 * pp] = t.v.x;
      u[2 * pp + 1] = t.v.y;
    }
    float f[2][NV];
    euler_flux_all<float, 2>(u, g1, f);
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) sF[((d * NP + pp) * Q + q) * TC + tc] = f32x2(f[d][2 * pp], f[d][2 * pp + 1]);
  }
  __syncthreads();
  if (!valid) return;

  // 3. volume and surface integrals of the pair
  f32x2 acc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l] = f32x2(0.0f);
  {
    f32x2 f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = sF[((0 * NP + p) * Q + q) * TC + tc];
    volume_dir<f32x2, 2, K, 0>(T, f, acc);
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = sF[((1 * NP + p) * Q + q) * TC + tc];
    volume_dir<f32x2, 2, K, 1>(T, f, acc);
  }
  auto surface = [&](auto sc) {
    constexpr int SD = decltype(sc)::value, DIR = SD >> 1, SS = SD & 1;
    const int e0 = a.m.sface[(size_t)SD * nc + c];
    f32x2 fq[QF];
    if (!((coarse >> SD) & 1)) {
#pragma unroll
      for (int q = 0; q < QF; ++q)
        fq[q] = f32x2(a.F[((size_t)v0 * QF + q) * nf + e0], a.F[((size_t)v1 * QF + q) * nf + e0]);
      surface_side<f32x2, 2, K, DIR, SS>(T, T.PW, T.PW, fq, f32x2(1.0f), acc);
    } else {
      // coarse side of a hanging face: NSUB sub-faces in quadrant order
      const f32x2 sub(1.0f / float(S::NSUB));
#pragma unroll
      for (int h = 0; h < S::NSUB; ++h) {
#pragma unroll
        for (int q = 0; q < QF; ++q)
          fq[q] = f32x2(a.F[((size_t)v0 * QF + q) * nf + e0 + h], a.F[((size_t)v1 * QF + q) * nf + e0 + h]);
        surface_side<f32x2, 2, K, DIR, SS>(T, T.PWH[h & 1], T.PWH[(h >> 1) & 1], fq, sub, acc);
      }
    }
  };
  surface(std::integral_constant<int, 0>{});
  surface(std::integral_constant<int, 1>{});
  surface(std::integral_constant<int, 2>{});
  surface(std::integral_constant<int, 3>{});

  // 4. epilogue out_o = ck_o sc acc + sum_r C[o][r] in_r, as in the scalar kernel
  const int pb = cell_problem(a.m, c);
  const float pre = a.pre_prob ? a.pre_prob[pb] : a.pre[a.m.level[c]];
  const float sc = pre * (a.dt ? float(a.dt[pb]) : 1.0f);
  const size_t i0 = (size_t)(v0 * N) * nc + c, i1 = (size_t)(v1 * N) * nc + c;
#pragma unroll
  for (int oo = 0; oo < MAX_OUT; ++oo) {
    if (oo >= a.n_out) break;
    const f32x2 ckv(a.ck[oo] * sc);
    f32x2 val[N];
#pragma unroll
    for (int j = 0; j < N; ++j) val[j] = ckv * acc[j];
#pragma unroll
    for (int r = 0; r < MAX_IN; ++r) {
      if (r >= a.n_in) break;
      const float cr = a.C[oo][r];
      if (cr == 0.0f) continue;
      const float* src = a.in[r];
      const f32x2 cr2(cr);
      if (src == a.U) {
#pragma unroll
        for (int j = 0; j < N; ++j) val[j] = fmac(cr2, w[j], val[j]);
      } else {
#pragma unroll
        for (int j = 0; j < N; ++j)
          val[j] = fmac(cr2, f32x2(src[i0 + (size_t)j * nc], src[i1 + (size_t)j * nc]), val[j]);
      }
    }
    float* dst = a.out[oo];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      dst[i0 + (size_t)j * nc] = val[j].v.x;
      dst[i1 + (size_t)j * nc] = val[j].v.y;
    }
  }
}

constexpr int X2_TC = 64;  // cells per block of the packed-pair cell kernel

template <int K>
cudaError_t launch_cell_x2(const void* pa, cudaStream_t s) {
  X2Args x;
  x.a = *static_cast<const StageArgs<float>*>(pa);
  if (x.a.m.ncells == 0) return cudaSuccess;
  constexpr int NT = sizeof(Tab1D<float>) / sizeof(float);
  static_assert(sizeof(Tab1D<f32x2>) == NT * sizeof(f32x2), "Tab1D layout");
  const float* src = reinterpret_cast<const float*>(&x.a.t1);
  f32x2* dst = reinterpret_cast<f32x2*>(&x.t2);
  for (int i = 0; i < NT; ++i) dst[i] = f32x2(src[i]);
  using XT = X2Tile<K, X2_TC>;
  cell_update_x2_kernel<K, X2_TC><<<(x.a.m.ncells + X2_TC - 1) / X2_TC, XT::THREADS, XT::SMEM, s>>>(x);
  return cudaGetLastError();
}

}  // namespace dgi
