// Tensor-core form of the cell kernel (FP32 state, 2D uniform meshes): the two
// contractions of a tile of 32 cells run on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), rows = (variable, cell):
//   MMA 1 (modal -> nodal)   D1[v,c][q] = sum_l W[v,c][l] phi_l(xi_q)
//   MMA 2 (volume - surface) D2[v,c][j] = sum_{d,q} f_d,v(q) dphi_j/dxi_d w_q
//                                        - sum_{side,q} sc fbar_v(q) phi_j w_q
// The pointwise Euler fluxes stay on the CUDA cores.  Near-FP32 accuracy with
// the TF32 tensor datapath by operand splitting: x = hi + lo with hi the
// nearest TF32 value of x and lo the nearest TF32 value of x - hi; the four
// products lo*lo + lo*hi + hi*lo + hi*hi accumulate in FP32 (four MMAs per
// contraction), leaving a relative error of about 2^-21 per product.
//
// Operands are staged in shared memory in the K-major, no-swizzle layout:
// 8-row x 16-byte core matrices stored contiguously, core matrices adjacent
// along K 128 bytes apart, 8-row groups (K/4)*128 bytes apart.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include <cstring>
#include <vector>

#include "dg_internal.h"
#include "dg_physics.cuh"

namespace dgi {

template <int K>
struct TcShape {
  using S = Shape<2, K>;
  static constexpr int TC = 32;                          // cells per tile
  static constexpr int M = 128;                          // rows: v * 32 + cell
  static constexpr int KP1 = (S::N + 7) / 8 * 8;         // K of MMA 1
  static constexpr int NQ = (S::Q + 15) / 16 * 16;       // N of MMA 1
  static constexpr int QP = (S::Q + 3) / 4 * 4;          // points, padded to groups of 4
  static constexpr int QFP = (S::QF + 3) / 4 * 4;        // face points, padded
  static constexpr int KV = 2 * QP;                      // volume part of K of MMA 2
  static constexpr int KP2 = KV + 4 * QFP;               // K of MMA 2 (multiple of 8)
  static constexpr int NJ = (S::N + 15) / 16 * 16;       // N of MMA 2
  static constexpr int B_FLOATS = 2 * NQ * KP1 + 2 * NJ * KP2;  // B1 hi|lo, B2 hi|lo
  // A1 hi|lo (the nodal values reuse it once MMA 1 is done), A2 hi|lo, B
  static constexpr int A1_FLOATS = 2 * M * KP1 > S::NV * S::Q * TC ? 2 * M * KP1 : S::NV * S::Q * TC;
  static constexpr int SMEM_FLOATS = A1_FLOATS + 2 * M * KP2 + B_FLOATS;
  static constexpr size_t SMEM = (size_t)SMEM_FLOATS * 4;
  static constexpr int TMEM_COLS = 32;
  static_assert(NQ + NJ <= TMEM_COLS, "tensor memory columns");
  static_assert(KP2 % 8 == 0 && KP1 % 8 == 0, "K steps of 8");
  static_assert((2 * M * KP1) % 4 == 0 && A1_FLOATS % 32 == 0, "16-byte alignment");
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

// D[0:M, 0:N) = A[0:M, 0:KP) B[0:N, 0:KP)^T with split operands, small
// products first: A_lo B_lo + A_lo B_hi + A_hi B_lo + A_hi B_hi; K steps of 8
template <int KP, int N, int M>
__device__ __forceinline__ void tc_gemm_split(uint32_t dtmem, const float* Ah, const float* Al,
                                              const float* Bh, const float* Bl) {
  constexpr uint32_t idesc = tc_idesc(N, M);
  const float* As[4] = {Al, Al, Ah, Ah};
  const float* Bs[4] = {Bl, Bh, Bl, Bh};
  uint32_t acc = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    // a K step of 8 is 256 bytes further: 16 in the descriptor's address
    // field (shared addresses stay below 2^18, so the field does not overflow)
    const uint64_t da = tc_desc(tc_smem(As[t]), KP), db = tc_desc(tc_smem(Bs[t]), KP);
#pragma unroll
    for (int ks = 0; ks < KP / 8; ++ks) {
      tc_mma(dtmem, da + (uint64_t)(16 * ks), db + (uint64_t)(16 * ks), idesc, acc);
      acc = 1;
    }
  }
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      tc_smem(mbar)));
}

// bounded wait on an mbarrier phase; false if it gave up
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(tc_smem(mbar)), "r"(parity));
  }
  return done != 0;
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
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(v[i]);
}

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

__device__ __forceinline__ void tc_st4(float* base, int off, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(base + off) = make_float4(a, b, c, d);
}

// split four consecutive K values of one row and store them (16-byte stores)
__device__ __forceinline__ void tc_put4(float* Ah, float* Al, int off, const float* x) {
  float h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) tc_split(x[i], h[i], l[i]);
  tc_st4(Ah, off, h[0], h[1], h[2], h[3]);
  tc_st4(Al, off, l[0], l[1], l[2], l[3]);
}

// Persistent CTAs of two warpgroups: warps v and v + 4 share the TMEM lane
// quarter (and A rows) of variable v and split each phase of a tile between
// them.  Each CTA keeps the B operands, its tensor memory and its barriers for
// all the tiles it processes (tile, tile + gridDim.x, ...), and loads the
// global inputs of its next tile while the current one is in flight.
template <int K>
__global__ void __launch_bounds__(256, 3) cell_update_tc_kernel(const StageArgs<float> a) {
  using S = Shape<2, K>;
  using T = TcShape<K>;
  constexpr int TC = T::TC, M = T::M, KP1 = T::KP1, KP2 = T::KP2, NQ = T::NQ, NJ = T::NJ;
  constexpr int N = S::N, Q = S::Q, QF = S::QF, NV = S::NV, QP = T::QP, QFP = T::QFP;
  constexpr int G1H = (KP1 / 4 + 1) / 2;  // 16-byte groups of an A1 row per half
  constexpr int WH = 4 * G1H;             // weights per thread
  constexpr int NG = QP / 4;              // groups of 4 volume points
  constexpr int QH = (Q + 1) / 2;         // nodal values per thread
  constexpr int JH = (N + 1) / 2;         // output coefficients per thread
  static_assert(2 * NG <= 8 && QH <= 16 && JH <= 16, "work split");
  extern __shared__ __align__(1024) float sm[];
  float* A1h = sm;
  float* A1l = A1h + M * KP1;
  float* sU = sm;  // [NV][Q][TC], over A1 once MMA 1 has read it
  float* A2h = sm + T::A1_FLOATS;
  float* A2l = A2h + M * KP2;
  float* B1h = A2l + M * KP2;
  float* B1l = B1h + NQ * KP1;
  float* B2h = B1l + NQ * KP1;
  float* B2l = B2h + NJ * KP2;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int v = warp & 3, half = warp >> 2;  // variable (TMEM lane quarter), half of the work
  const int nc = a.m.ncells, nf = a.m.nfaces;
  const int ntiles = (nc + TC - 1) / TC;
  const int row = v * TC + lane;

  for (int i = threadIdx.x; i < T::B_FLOATS; i += 256) B1h[i] = __ldg(a.tcB + i);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[1])));
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
  const uint32_t trow = (uint32_t)(v * 32) << 16;
  const float g1 = (float)a.gamma - 1.0f;
  bool ok = true;
  uint32_t phase = 0;

  // this thread's share of a tile's global inputs: weights l = half*WH + i of
  // (v, c) and the fluxes of sides 2*half, 2*half+1; loaded a tile ahead
  float wn[WH], xn[2][QF];
  auto load_tile = [&](int t) {
    const int cc = t * TC + lane;
    const bool in = t < ntiles && cc < nc;
#pragma unroll
    for (int i = 0; i < WH; ++i) {
      const int l = half * WH + i;
      wn[i] = (in && l < N) ? a.U[(size_t)(v * N + l) * nc + cc] : 0.0f;
    }
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int e = in ? a.m.sface[(size_t)(2 * half + s2) * nc + cc] : 0;
#pragma unroll
      for (int q = 0; q < QF; ++q) xn[s2][q] = in ? a.F[((size_t)v * QF + q) * nf + e] : 0.0f;
    }
  };
  load_tile(blockIdx.x);

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, phase ^= 1u) {
    const int c = tile * TC + lane;
    const bool valid = c < nc;
    // weights -> A1 (a padding cell gets the unit density state)
    {
      float w[WH];
#pragma unroll
      for (int i = 0; i < WH; ++i) w[i] = wn[i];
      if (!valid && v == 0 && half == 0) w[0] = 1.0f;
#pragma unroll
      for (int g = 0; g < G1H; ++g)
        if ((half * G1H + g) * 4 < KP1)
          tc_put4(A1h, A1l, tc_off(row, (half * G1H + g) * 4, KP1), &w[4 * g]);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_gemm_split<KP1, NQ, M>(tmem, A1h, A1l, B1h, B1l);
      tc_commit(&mbar[0]);
    }
    // while MMA 1 runs: face fluxes of two sides -> surface part of A2
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      float x[QFP];
#pragma unroll
      for (int q = 0; q < QFP; ++q) x[q] = q < QF ? xn[s2][q] : 0.0f;
#pragma unroll
      for (int g = 0; g < QFP / 4; ++g)
        tc_put4(A2h, A2l, tc_off(row, T::KV + (2 * half + s2) * QFP + 4 * g, KP2), &x[4 * g]);
    }
    load_tile(tile + gridDim.x);
    // while MMA 1 runs: the stage combination of the inputs (all but the RHS
    // term) for coefficients j = half*JH + jj
    float base[MAX_OUT][JH];
    float scale = 0.0f;
    if (valid) {
      const int pb = cell_problem(a.m, c);
      const float pv = a.pre_prob ? a.pre_prob[pb] : a.pre[a.m.level[c]];
      scale = pv * (a.dt ? (float)a.dt[pb] : 1.0f);
    }
#pragma unroll
    for (int oo = 0; oo < MAX_OUT; ++oo)
#pragma unroll
      for (int jj = 0; jj < JH; ++jj) base[oo][jj] = 0.0f;
    for (int r = 0; r < a.n_in; ++r) {
      float xr[JH];
#pragma unroll
      for (int jj = 0; jj < JH; ++jj) {
        const int j = half * JH + jj;
        xr[jj] = (valid && j < N) ? a.in[r][(size_t)(v * N + j) * nc + c] : 0.0f;
      }
#pragma unroll
      for (int oo = 0; oo < MAX_OUT; ++oo) {
        const float cr = a.C[oo][r];
#pragma unroll
        for (int jj = 0; jj < JH; ++jj) base[oo][jj] += cr * xr[jj];
      }
    }
    ok = tc_wait(&mbar[0], phase) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;");
    {
      float u[16];
      tc_ld16(tmem + trow, u);
      // this thread saw MMA 1 complete, so its reads of A1 are over: sU may overwrite A1
#pragma unroll
      for (int i = 0; i < QH; ++i) {
        const int q = half * QH + i;
        const float val = half ? (QH + i < 16 ? u[QH + i] : 0.0f) : u[i];
        if (q < Q) sU[(v * Q + q) * TC + lane] = val;
      }
    }
    __syncthreads();
    // Euler flux in direction d at points 4g..4g+3 (task = warp) -> volume part of A2
    if (warp < 2 * NG) {
      const int d = warp & 1, g = warp >> 1;
      float f[NV][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int q = 4 * g + i;
        float u[NV], fd[NV];
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) u[vv] = q < Q ? sU[(vv * Q + q) * TC + lane] : (vv == 0 ? 1.0f : 0.0f);
        if (d == 0)
          euler_flux<float, 2>(u, 0, g1, fd);
        else
          euler_flux<float, 2>(u, 1, g1, fd);
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) f[vv][i] = q < Q ? fd[vv] : 0.0f;
      }
#pragma unroll
      for (int vv = 0; vv < NV; ++vv)
        tc_put4(A2h, A2l, tc_off(vv * TC + lane, d * QP + 4 * g, KP2), f[vv]);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (threadIdx.x == 0) {
      tc_gemm_split<KP2, NJ, M>(tmem + NQ, A2h, A2l, B2h, B2l);
      tc_commit(&mbar[1]);
    }
    ok = tc_wait(&mbar[1], phase) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float acc[16];
    tc_ld16(tmem + trow + NQ, acc);
    if (valid && ok) {
#pragma unroll
      for (int oo = 0; oo < MAX_OUT; ++oo)
        if (oo < a.n_out) {
          const float ckv = a.ck[oo] * scale;
#pragma unroll
          for (int jj = 0; jj < JH; ++jj) {
            const int j = half * JH + jj;
            const float rhs = half ? (JH + jj < 16 ? acc[JH + jj] : 0.0f) : acc[jj];
            if (j < N) a.out[oo][(size_t)(v * N + j) * nc + c] = base[oo][jj] + ckv * rhs;
          }
        }
    }
    // all warps are done with MMA 2's operands and results before the next
    // tile; a wait that gave up anywhere ends the CTA's work
    asm volatile("tcgen05.fence::before_thread_sync;");
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) break;
  }
  if (!ok && threadIdx.x == 0) atomicOr(a.status, 1 << DG_ERR_TIMEOUT_BIT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
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

template <int K>
struct TcGrid {
  static inline int ctas = 0;  // resident CTAs on the whole device (set by prepare_cell_tc)
};

template <int K>
cudaError_t launch_cell_tc(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const StageArgs<float>*>(pa);
  using T = TcShape<K>;
  if (a.m.ncells == 0) return cudaSuccess;
  const int ntiles = (a.m.ncells + T::TC - 1) / T::TC;
  const int grid = TcGrid<K>::ctas > 0 && TcGrid<K>::ctas < ntiles ? TcGrid<K>::ctas : ntiles;
  cell_update_tc_kernel<K><<<grid, 256, T::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int K>
cudaError_t prepare_cell_tc() {
  cudaError_t e = cudaFuncSetAttribute(cell_update_tc_kernel<K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TcShape<K>::SMEM);
  if (e != cudaSuccess) return e;
  // all of the unified L1/shared storage as shared memory: several CTAs per SM
  e = cudaFuncSetAttribute(cell_update_tc_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  // resident CTAs per SM from the kernel's registers and shared memory
  int dev = 0, sms = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0;
  cudaFuncAttributes fa;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  if ((e = cudaFuncGetAttributes(&fa, cell_update_tc_kernel<K>)) != cudaSuccess) return e;
  const int by_smem = smem_sm / (int)(TcShape<K>::SMEM + fa.sharedSizeBytes + smem_rsv);
  const int by_regs = regs_sm / ((fa.numRegs > 0 ? fa.numRegs : 1) * 256);
  int per_sm = by_smem < by_regs ? by_smem : by_regs;
  if (per_sm > 8) per_sm = 8;  // 2048 threads per SM
  TcGrid<K>::ctas = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

}  // namespace dgi
