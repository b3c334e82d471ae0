// Tensor-core form of the cell kernel (2D uniform meshes, k = 1..3): the two
// contractions of the cell update (paper Sec. 2.4, eqs. dg_term2, dg_term3)
// run on the 5th-generation tensor cores (tcgen05.mma, accumulators in
// tensor memory) for tiles of 128 cells, one MMA row (TMEM lane) per cell:
//   MMA 1, per variable v (modal -> nodal)
//       D1_v[c][q] = sum_l W[v][l][c] phi_l(xi_q)
//   MMA 2, per variable v (volume - surface)
//       D2_v[c][j] = sum_{d,q} f_d,v(q) dphi_j/dxi_d w_q - sum_{side,q} sc fbar_v(q) phi_j w_q
// The pointwise Euler fluxes stay on the CUDA cores.  Because a TMEM lane
// holds every variable of its cell, the four threads of a cell read the
// nodal values they need straight from tensor memory (no exchange through
// shared memory).
//
// Two state forms share the kernel: an FP32 state (DG_FP32_TC) and the
// mixed mode's FP64 state with its right-hand side in perturbation form
// (DG_MIXED_TC; dg_mixed.cuh): there MMA 1 sees the perturbation weights,
// the fluxes are f(ubar + du) - f(ubar) and the face values G (+ D).
//
// Near-FP32 accuracy with the TF32 tensor datapath by operand splitting:
// x = hi + lo with hi the nearest TF32 value of x and lo the nearest TF32
// value of x - hi.  Three products per contraction, lo*hi + hi*lo + hi*hi,
// accumulate in FP32; the dropped lo*lo term and the rounding of lo are
// each below 2^-22 of |a||b| per product.
//
// Operands are staged in shared memory in the K-major, no-swizzle layout:
// 8-row x 16-byte core matrices stored contiguously, core matrices adjacent
// along K 128 bytes apart, 8-row groups (K/4)*128 bytes apart.
//
// Work split: 512 threads per CTA, four per cell; thread t of a cell (the
// warp's index over 4) handles variable t for the weights and the epilogue,
// volume points PT*t .. PT*t+PT-1 for the fluxes, and side t for the face
// values.  One CTA per SM (200 KB of shared memory at k = 3), persistent over
// tiles; the inputs of a CTA's next tile are loaded while MMA 1 runs.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "dg_convert.cuh"
#include "dg_internal.h"
#include "dg_mixed.cuh"
#include "dg_physics.cuh"

namespace dgi {

template <int K>
struct TcShape {
  using S = Shape<2, K>;
  static constexpr int TM = 128;                         // cells per tile = MMA rows = TMEM lanes
  static constexpr int THREADS = 512;                    // four threads per cell
  static constexpr int PT = (S::Q + 3) / 4;              // volume points per thread
  static constexpr int QP = 4 * PT;                      // volume points, padded
  static constexpr int KP1 = (S::N + 7) / 8 * 8;         // K of MMA 1 (coefficients, steps of 8)
  static constexpr int NQ = 16;                          // N of MMA 1 (points)
  static constexpr int QFP = 4;                          // face points per side, padded
  static constexpr int KV = 2 * QP;                      // volume part of K of MMA 2
  static constexpr int KP2 = KV + 4 * QFP;               // K of MMA 2
  static constexpr int NJ = 16;                          // N of MMA 2 (coefficients)
  static constexpr int A1_BLK = TM * KP1;                // floats of one (variable, hi|lo) block
  static constexpr int A2_BLK = TM * KP2;
  static constexpr int A2_FLOATS = 2 * S::NV * A2_BLK;   // [variable][hi|lo][TM x KP2]
  static constexpr int A1_OFF = 2 * 2 * A2_BLK;          // A1 over the A2 blocks of variables 2, 3
  static constexpr int B_FLOATS = 2 * NQ * KP1 + 2 * NJ * KP2;  // B1 hi|lo, B2 hi|lo
  static constexpr int SMEM_FLOATS = A2_FLOATS + B_FLOATS;
  static constexpr size_t SMEM = (size_t)SMEM_FLOATS * 4;
  static constexpr int D1_COL = 0;                       // TMEM columns of D1_v: 16 v ..
  static constexpr int D2_COL = 16 * S::NV;              // and of D2_v: 64 + 16 v ..
  static constexpr int TMEM_COLS = 128;
  static_assert(S::NV == 4 && QP <= NQ && S::N <= NJ && S::QF <= QFP, "2D shapes");
  static_assert(2 * S::NV * A1_BLK <= A2_FLOATS - A1_OFF, "A1 fits over the A2 blocks of variables 2, 3");
  static_assert(KP1 % 8 == 0 && KP2 % 8 == 0, "K steps of 8");
  static_assert(D2_COL + 16 * S::NV <= TMEM_COLS, "tensor memory columns");
  static_assert(SMEM + 8 * 1024 <= 227 * 1024, "shared memory of one CTA");
};

// float offset of element (r, k) in the core-matrix layout of a tile with KP columns
__host__ __device__ __forceinline__ int tc_off(int r, int k, int KP) {
  return ((r >> 3) * (KP >> 2) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint32_t tc_smem(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, int KP) {
  const uint32_t lbo = 128, sbo = (uint32_t)(KP / 4) * 128;
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; base offset 0; no swizzle
  return d;
}

// kind::tf32, D F32, A/B TF32 K-major, N x M tile
__host__ __device__ constexpr uint32_t tc_idesc(int n, int m) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// The four per-variable contractions D_v = A_v B^T (v = 0..3; D_v at TMEM
// column dcol + 16 v, A_v hi|lo at Ab + 2 v blk, Ab + (2 v + 1) blk) with
// split operands, issued so that consecutive multiplies accumulate into
// different variables' columns (four independent chains)
template <int KP>
__device__ __forceinline__ void tc_gemm3_x4(uint32_t dcol, const float* Ab, int blk, const float* Bh,
                                            const float* Bl) {
  constexpr uint32_t idesc = tc_idesc(16, 128);
  uint64_t dah[4], dal[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    dah[v] = tc_desc(tc_smem(Ab + (2 * v) * blk), KP);
    dal[v] = tc_desc(tc_smem(Ab + (2 * v + 1) * blk), KP);
  }
  const uint64_t dbh = tc_desc(tc_smem(Bh), KP), dbl = tc_desc(tc_smem(Bl), KP);
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int ks = 0; ks < KP / 8; ++ks)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint64_t da = (t == 0 ? dal[v] : dah[v]) + (uint64_t)(16 * ks);
        const uint64_t db = (t == 1 ? dbl : dbh) + (uint64_t)(16 * ks);
        tc_mma(dcol + 16 * v, da, db, idesc, (t == 0 && ks == 0) ? 0u : 1u);
      }
}

// D_v = A_v B^T for one variable (D_v at TMEM column dcol, A_v hi|lo at Ah, Al)
template <int KP>
__device__ __forceinline__ void tc_gemm3(uint32_t dcol, const float* Ah, const float* Al, const float* Bh,
                                         const float* Bl) {
  constexpr uint32_t idesc = tc_idesc(16, 128);
  const uint64_t dah = tc_desc(tc_smem(Ah), KP), dal = tc_desc(tc_smem(Al), KP);
  const uint64_t dbh = tc_desc(tc_smem(Bh), KP), dbl = tc_desc(tc_smem(Bl), KP);
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int ks = 0; ks < KP / 8; ++ks) {
      const uint64_t da = (t == 0 ? dal : dah) + (uint64_t)(16 * ks);
      const uint64_t db = (t == 1 ? dbl : dbh) + (uint64_t)(16 * ks);
      tc_mma(dcol, da, db, idesc, (t == 0 && ks == 0) ? 0u : 1u);
    }
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      tc_smem(mbar)));
}

// bounded wait on an mbarrier phase; false if it gave up after `limit` polls
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t parity, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(tc_smem(mbar)), "r"(parity));
  }
  return done != 0;
}

// tensor memory -> registers: lane of this thread, columns taddr .. (+1, +4, +16)
__device__ __forceinline__ float tc_ld1(uint32_t taddr) {
  uint32_t v;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr));
  return __uint_as_float(v);
}

__device__ __forceinline__ void tc_ld4(uint32_t taddr, float* out) {
  uint32_t v[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = __uint_as_float(v[i]);
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* out) {
  uint32_t v[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(v[i]);
}

__device__ __forceinline__ void tc_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tc_round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x = hi + lo + O(2^-22 |x|), both parts TF32 values
__device__ __forceinline__ void tc_split(float x, float& hi, float& lo) {
  hi = tc_round_tf32(x);
  lo = tc_round_tf32(x - hi);
}

// split four consecutive K values of one row and store them (16-byte stores)
__device__ __forceinline__ void tc_put4(float* Ah, float* Al, int off, const float* x) {
  float h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) tc_split(x[i], h[i], l[i]);
  *reinterpret_cast<float4*>(Ah + off) = make_float4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<float4*>(Al + off) = make_float4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void tc_put1(float* Ah, float* Al, int off, float x) {
  float h, l;
  tc_split(x, h, l);
  Ah[off] = h;
  Al[off] = l;
}

template <bool MIXED>
using TcArgs = typename std::conditional<MIXED, MixedArgs, StageArgs<float>>::type;

__host__ __device__ __forceinline__ const StageArgs<float>& tc_stage(const StageArgs<float>& a) { return a; }
__host__ __device__ __forceinline__ const StageArgs<double>& tc_stage(const MixedArgs& x) { return x.a; }
// gamma - 1 in FP32, rounded as (float)gamma - 1.0f on the host
__host__ __device__ __forceinline__ float tc_g1(const StageArgs<float>& a) { return a.gm1; }
__host__ __device__ __forceinline__ float tc_g1(const MixedArgs& x) { return x.g1f; }

template <int K, bool MIXED>
__global__ void __launch_bounds__(512, 1) cell_tc_kernel(const TcArgs<MIXED> x) {
  using S = Shape<2, K>;
  using T = TcShape<K>;
  constexpr int N = S::N, Q = S::Q, QF = S::QF, NV = S::NV;
  constexpr int TM = T::TM, PT = T::PT, QP = T::QP, KP1 = T::KP1, KP2 = T::KP2, NQ = T::NQ, NJ = T::NJ;
  constexpr int QFP = T::QFP;
  const auto& a = tc_stage(x);
  extern __shared__ __align__(1024) float sm[];
  float* const A2 = sm;               // block (v, h) at (2 v + h) A2_BLK
  float* const A1 = sm + T::A1_OFF;   // block (v, h) at (2 v + h) A1_BLK, over A2 of variables 2, 3
  float* const B1h = sm + T::A2_FLOATS;
  float* const B1l = B1h + NQ * KP1;
  float* const B2h = B1l + NQ * KP1;
  float* const B2l = B2h + NJ * KP2;
  // mbar[0]: MMA 1 done; mbar[1 + v]: MMA 2 of variable v (and those before it) done
  __shared__ __align__(8) uint64_t mbar[5];
  __shared__ uint32_t tmem_base;
  // mixed: reference state and residual of every (variable, cell) of the tile
  __shared__ float sRef[MIXED ? NV * TM : 1], sRes[MIXED ? NV * TM : 1];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row = ((warp & 3) << 5) | lane;  // the cell within the tile (TMEM lane)
  const int t = warp >> 2;                   // variable, point group and side of this thread
  const int nc = a.m.ncells, nf = a.m.nfaces;
  const int ntiles = (nc + TM - 1) / TM;
  const bool hook = a.tc_hook != 0 && blockIdx.x == 0;
  const int limit = hook ? (1 << 12) : (1 << 24);

  for (int i = tid; i < T::B_FLOATS; i += T::THREADS) B1h[i] = __ldg(x.tcB + i);
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[i])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem(&tmem_base)),
                 "r"(T::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lane quarter
  const float g1 = tc_g1(x);

  // This thread's inputs of a tile, loaded a tile ahead: the weights of
  // variable t (FP32: as stored, a padding cell gets the unit density state;
  // mixed: the perturbation weights l >= 1, the mean as reference + residual)
  // and the face values of side t for every variable.
  float wn[KP1], xn[NV][QFP], ubn = 0.0f, resn = 0.0f;
  auto load_tile = [&](int tt) {
    const int cc = tt * TM + row;
    const bool in = tt < ntiles && cc < nc;
    const size_t i0 = (size_t)t * N * nc + cc;
#pragma unroll
    for (int l = 0; l < KP1; ++l) wn[l] = 0.0f;
    if constexpr (!MIXED) {
#pragma unroll
      for (int l = 0; l < N; ++l) wn[l] = in ? a.U[i0 + (size_t)l * nc] : 0.0f;
      if (!in && t == 0) wn[0] = 1.0f;
    } else {
      ubn = (!in && t == 0) ? 1.0f : 0.0f;
      resn = 0.0f;
      if (in) {
        float hi, lo;
        if (x.wf_mode == 2) {
          hi = x.Wf[i0];
          lo = x.Wlo[(size_t)t * nc + cc];
        } else {
          df_split(a.U[i0], hi, lo);
          if (x.wf_mode == 1) {
            x.Wf[i0] = hi;
            x.Wlo[(size_t)t * nc + cc] = lo;
          }
        }
        mixed_mean_split(hi, lo, x.R, i0, ubn, resn);
#pragma unroll
        for (int l = 1; l < N; ++l) {
          const size_t il = i0 + (size_t)l * nc;
          float wl;
          if (x.wf_mode == 2) {
            wl = x.Wf[il];
          } else {
            wl = f32_round(a.U[il]);
            if (x.wf_mode == 1) x.Wf[il] = wl;
          }
          wn[l] = x.R ? wl + x.R[il] : wl;
        }
      }
    }
    const int e = in ? a.m.sface[(size_t)t * nc + cc] : 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float dv = 0.0f;
      if constexpr (MIXED) dv = (in && !(t & 1)) ? x.D[(size_t)v * nf + e] : 0.0f;
#pragma unroll
      for (int q = 0; q < QFP; ++q) {
        if constexpr (MIXED) xn[v][q] = (in && q < QF) ? x.G[((size_t)v * QF + q) * nf + e] + dv : 0.0f;
        else xn[v][q] = (in && q < QF) ? a.F[((size_t)v * QF + q) * nf + e] : 0.0f;
      }
    }
  };
  load_tile(blockIdx.x);

  bool ok = true;
  uint32_t phase = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, phase ^= 1u) {
    const int c = tile * TM + row;
    const bool valid = c < nc;
    // ---- A. weights of variable t -> A1; face values of variables 0, 1 -> A2
    // (the A2 blocks of variables 2, 3 hold A1 until MMA 1 is done).  The
    // previous tile's last MMA-2 chain (and so every one before it) must be
    // done reading A2 first: this thread waited only for its own variable's.
    if (tile != (int)blockIdx.x) ok = tc_wait(&mbar[NV], phase ^ 1u, limit) && ok;
    float wcur[MIXED ? 1 : N];
    if constexpr (!MIXED) {
#pragma unroll
      for (int l = 0; l < N; ++l) wcur[l] = wn[l];
    } else {
      sRef[t * TM + row] = ubn;
      sRes[t * TM + row] = resn;
    }
#pragma unroll
    for (int g = 0; g < KP1 / 4; ++g)
      tc_put4(A1 + (2 * t) * T::A1_BLK, A1 + (2 * t + 1) * T::A1_BLK, tc_off(row, 4 * g, KP1), &wn[4 * g]);
    float xlate[2][QFP];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      tc_put4(A2 + (2 * v) * T::A2_BLK, A2 + (2 * v + 1) * T::A2_BLK, tc_off(row, T::KV + 4 * t, KP2), xn[v]);
#pragma unroll
      for (int q = 0; q < QFP; ++q) xlate[v][q] = xn[2 + v][q];
    }
    asm volatile("fence.proxy.async.shared::cta;");
    // all stores of the tile are visible; a failed wait of the previous tile
    // (carried in ok) ends the CTA's work
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    if (tid == 0 && !(hook && tile == (int)blockIdx.x)) {
      tc_gemm3_x4<KP1>(tmem + T::D1_COL, A1, T::A1_BLK, B1h, B1l);
      tc_commit(&mbar[0]);
    }
    // while MMA 1 runs: the inputs of the next tile
    load_tile(tile + gridDim.x);
    ok = tc_wait(&mbar[0], phase, limit) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;");

    // ---- B. nodal values at this thread's points (tensor memory) -> fluxes -> A2
    float u[NV][PT];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if constexpr (PT == 4) {
        tc_ld4(tl + T::D1_COL + 16 * v + 4 * t, u[v]);
      } else {
#pragma unroll
        for (int i = 0; i < PT; ++i) u[v][i] = tc_ld1(tl + T::D1_COL + 16 * v + PT * t + i);
      }
    }
    tc_ld_wait();
    float fx[NV][PT], fy[NV][PT];
    {
      float ub[NV], res[NV];
      if constexpr (MIXED) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          ub[v] = sRef[v * TM + row];
          res[v] = sRes[v * TM + row];
        }
      }
#pragma unroll
      for (int i = 0; i < PT; ++i) {
        const bool live = PT * t + i < Q;
        if constexpr (!MIXED) {
          float uu[NV], f[2][NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) uu[v] = live ? u[v][i] : (v == 0 ? 1.0f : 0.0f);
          euler_flux_all<float, 2>(uu, g1, f);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            fx[v][i] = live ? f[0][v] : 0.0f;
            fy[v][i] = live ? f[1][v] : 0.0f;
          }
        } else {
          const RefState<float, 2> rs = ref_state<float, 2>(ub, g1);
          float du[NV], f0[NV], f1[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) du[v] = live ? u[v][i] + res[v] : 0.0f;
          const Pert<float, 2> pq = perturb<float, 2>(rs, du, g1);
          euler_dflux<float, 2>(rs, du, pq, 0, f0);
          euler_dflux<float, 2>(rs, du, pq, 1, f1);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            fx[v][i] = live ? f0[v] : 0.0f;
            fy[v][i] = live ? f1[v] : 0.0f;
          }
        }
      }
    }
    // MMA 1 is complete (this thread saw its barrier), so A1 may be overwritten
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float* Ah = A2 + (2 * v) * T::A2_BLK;
      float* Al = A2 + (2 * v + 1) * T::A2_BLK;
      if constexpr (PT == 4) {
        tc_put4(Ah, Al, tc_off(row, 4 * t, KP2), fx[v]);
        tc_put4(Ah, Al, tc_off(row, QP + 4 * t, KP2), fy[v]);
      } else {
#pragma unroll
        for (int i = 0; i < PT; ++i) {
          tc_put1(Ah, Al, tc_off(row, PT * t + i, KP2), fx[v][i]);
          tc_put1(Ah, Al, tc_off(row, QP + PT * t + i, KP2), fy[v][i]);
        }
      }
      if (v >= 2) tc_put4(Ah, Al, tc_off(row, T::KV + 4 * t, KP2), xlate[v - 2]);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    const bool all_ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!all_ok) {
      ok = false;
      break;
    }
    if (tid == 0) {
      // one chain per variable, each with its own barrier: the threads of
      // variable v start their epilogue once chain v is done
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        tc_gemm3<KP2>(tmem + T::D2_COL + 16 * v, A2 + (2 * v) * T::A2_BLK, A2 + (2 * v + 1) * T::A2_BLK, B2h, B2l);
        tc_commit(&mbar[1 + v]);
      }
    }

    // ---- C. while MMA 2 runs: the stage combination of the inputs for
    // variable t (all but the right-hand side term)
    const size_t iv = (size_t)t * N * nc + c;
    if constexpr (!MIXED) {
      float base[MAX_OUT][N];
#pragma unroll
      for (int oo = 0; oo < MAX_OUT; ++oo)
#pragma unroll
        for (int j = 0; j < N; ++j) base[oo][j] = 0.0f;
      float scale = 0.0f;
      if (valid) {
        const int pb = cell_problem(a.m, c);
        scale = (a.pre_prob ? a.pre_prob[pb] : a.pre[a.m.level[c]]) * (a.dt ? (float)a.dt[pb] : 1.0f);
#pragma unroll
        for (int r = 0; r < MAX_IN; ++r) {
          if (r >= a.n_in) break;
          const float* src = a.in[r];
          const bool own = src == a.U;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const float xr = own ? wcur[j] : src[iv + (size_t)j * nc];
#pragma unroll
            for (int oo = 0; oo < MAX_OUT; ++oo) base[oo][j] += a.C[oo][r] * xr;
          }
        }
      }
      ok = tc_wait(&mbar[1 + t], phase, limit) && ok;
      asm volatile("tcgen05.fence::after_thread_sync;");
      float acc[16];
      tc_ld16(tl + T::D2_COL + 16 * t, acc);
      tc_ld_wait();
      if (valid && ok) {
#pragma unroll
        for (int oo = 0; oo < MAX_OUT; ++oo) {
          if (oo >= a.n_out) break;
          const float ckv = a.ck[oo] * scale;
#pragma unroll
          for (int j = 0; j < N; ++j) a.out[oo][iv + (size_t)j * nc] = base[oo][j] + ckv * acc[j];
        }
      }
    } else {
      float base[N];
#pragma unroll
      for (int j = 0; j < N; ++j) base[j] = 0.0f;
      if (x.delta && valid) {
        for (int r = 0; r < x.n_inR; ++r) {
          const float cr = x.Cf[r];
#pragma unroll
          for (int j = 0; j < N; ++j) base[j] += cr * x.inR[r][iv + (size_t)j * nc];
        }
      }
      ok = tc_wait(&mbar[1 + t], phase, limit) && ok;
      asm volatile("tcgen05.fence::after_thread_sync;");
      float acc[16];
      tc_ld16(tl + T::D2_COL + 16 * t, acc);
      tc_ld_wait();
      if (valid && ok) {
        const int pb = cell_problem(a.m, c);
        const double pre = a.pre_prob ? a.pre_prob[pb] : a.pre[a.m.level[c]];
        const double dtv = a.dt ? a.dt[pb] : 1.0;
        if (x.delta) {
          const float sc = x.ckf * f32_round(dtv * pre);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const size_t idx = iv + (size_t)j * nc;
            const float val = base[j] + sc * acc[j];
            if (x.outR) x.outR[idx] = val;
            else a.out[0][idx] = a.U[idx] + f64_exact(val);
          }
        } else {
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const size_t idx = iv + (size_t)j * nc;
            const double rhs = pre * f64_exact(acc[j]);
            for (int oo = 0; oo < a.n_out; ++oo) {
              double val = a.ck[oo] * dtv * rhs;
              for (int r = 0; r < a.n_in; ++r) {
                const double cr = a.C[oo][r];
                if (cr != 0.0) val += cr * a.in[r][idx];
              }
              a.out[oo][idx] = val;
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  // a wait that gave up anywhere: the CTA stopped early; report it.  No
  // tensor-core work of this CTA is in flight unless a multiply it issued
  // never completed.
  ok = __syncthreads_and(ok) != 0;
  if (!ok && tid == 0) atomicOr(a.status, 1 << DG_ERR_TIMEOUT_BIT);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T::TMEM_COLS));
}

// host: B operands (hi | lo, core-matrix layout) from the FP64 tables
template <int K>
void fill_tc_tables(const std::vector<double>& Tab, std::vector<float>& out) {
  using S = Shape<2, K>;
  using T = TcShape<K>;
  out.assign(T::B_FLOATS, 0.0f);
  float* B1h = out.data();
  float* B1l = B1h + T::NQ * T::KP1;
  float* B2h = B1l + T::NQ * T::KP1;
  float* B2l = B2h + T::NJ * T::KP2;
  auto tf32 = [](float f) {  // nearest TF32 value (ties away from zero)
    uint32_t b;
    std::memcpy(&b, &f, 4);
    b = (b + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
  };
  auto split = [&](double x, float& hi, float& lo) {
    hi = tf32((float)x);
    lo = tf32((float)(x - (double)hi));
  };
  for (int q = 0; q < S::Q; ++q)
    for (int l = 0; l < S::N; ++l) {
      float hi, lo;
      split(Tab[S::OFF_PHI + q * S::N + l], hi, lo);
      B1h[tc_off(q, l, T::KP1)] = hi;
      B1l[tc_off(q, l, T::KP1)] = lo;
    }
  for (int j = 0; j < S::N; ++j) {
    for (int d = 0; d < 2; ++d)
      for (int q = 0; q < S::Q; ++q) {
        float hi, lo;
        split(Tab[S::OFF_DPHIW + (d * S::Q + q) * S::N + j], hi, lo);
        B2h[tc_off(j, d * T::QP + q, T::KP2)] = hi;
        B2l[tc_off(j, d * T::QP + q, T::KP2)] = lo;
      }
    for (int sd = 0; sd < 4; ++sd)
      for (int q = 0; q < S::QF; ++q) {
        const double sc = (sd & 1) ? 1.0 : -1.0;  // outward normal sign of the side
        float hi, lo;
        split(-sc * Tab[S::OFF_PHIFW + ((sd * S::NVAR + 0) * S::QF + q) * S::N + j], hi, lo);
        B2h[tc_off(j, T::KV + sd * T::QFP + q, T::KP2)] = hi;
        B2l[tc_off(j, T::KV + sd * T::QFP + q, T::KP2)] = lo;
      }
  }
}

template <int K, bool MIXED>
struct TcGrid {
  static inline int ctas = 0;  // resident CTAs on the whole device (set by prepare_cell_tc)
};

template <int K, bool MIXED>
cudaError_t launch_cell_tc(const void* pa, cudaStream_t s) {
  const auto& x = *static_cast<const TcArgs<MIXED>*>(pa);
  using T = TcShape<K>;
  const int nc = tc_stage(x).m.ncells;
  if (nc == 0) return cudaSuccess;
  const int ntiles = (nc + T::TM - 1) / T::TM;
  const int ctas = TcGrid<K, MIXED>::ctas;
  const int grid = ctas > 0 && ctas < ntiles ? ctas : ntiles;
  cell_tc_kernel<K, MIXED><<<grid, T::THREADS, T::SMEM, s>>>(x);
  return cudaGetLastError();
}

template <int K, bool MIXED>
cudaError_t prepare_cell_tc() {
  cudaError_t e = cudaFuncSetAttribute(cell_tc_kernel<K, MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TcShape<K>::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(cell_tc_kernel<K, MIXED>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  // one persistent CTA per resident slot: the occupancy calculator's count
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell_tc_kernel<K, MIXED>, TcShape<K>::THREADS,
                                                         TcShape<K>::SMEM)) != cudaSuccess)
    return e;
  TcGrid<K, MIXED>::ctas = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

}  // namespace dgi
