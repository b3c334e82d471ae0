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

#include "dg_internal.h"
#include "dg_physics.cuh"

namespace dgi {

template <int K>
struct TcShape {
  using S = Shape<2, K>;
  static constexpr int TC = 32;                          // cells per CTA
  static constexpr int M = 128;                          // rows: v * 32 + cell
  static constexpr int KP1 = (S::N + 7) / 8 * 8;         // K of MMA 1
  static constexpr int NQ = (S::Q + 15) / 16 * 16;       // N of MMA 1
  static constexpr int KV = 2 * S::Q;                    // volume part of K of MMA 2
  static constexpr int KS = 4 * S::QF;                   // surface part
  static constexpr int KP2 = (KV + KS + 7) / 8 * 8;      // K of MMA 2
  static constexpr int NJ = (S::N + 15) / 16 * 16;       // N of MMA 2
  static constexpr int B_FLOATS = 2 * NQ * KP1 + 2 * NJ * KP2;  // B1 hi|lo, B2 hi|lo
  static constexpr int SMEM_FLOATS = 2 * M * KP1 + 2 * M * KP2 + B_FLOATS + S::NV * S::Q * TC;
  static constexpr size_t SMEM = (size_t)SMEM_FLOATS * 4;
  static constexpr int TMEM_COLS = 32;
  static_assert(NQ + NJ <= TMEM_COLS, "tensor memory columns");
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
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int ks = 0; ks < KP / 8; ++ks) {
      tc_mma(dtmem, tc_desc(tc_smem(As[t]) + ks * 256, KP), tc_desc(tc_smem(Bs[t]) + ks * 256, KP),
             idesc, acc);
      acc = 1;
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

template <int K>
__global__ void __launch_bounds__(128) cell_update_tc_kernel(const StageArgs<float> a) {
  using S = Shape<2, K>;
  using T = TcShape<K>;
  constexpr int TC = T::TC, M = T::M, KP1 = T::KP1, KP2 = T::KP2, NQ = T::NQ, NJ = T::NJ;
  constexpr int N = S::N, Q = S::Q, QF = S::QF, NV = S::NV;
  extern __shared__ __align__(1024) float sm[];
  float* A1h = sm;
  float* A1l = A1h + M * KP1;
  float* A2h = A1l + M * KP1;
  float* A2l = A2h + M * KP2;
  float* Bs = A2l + M * KP2;  // B1h | B1l | B2h | B2l
  float* B1h = Bs;
  float* B1l = B1h + NQ * KP1;
  float* B2h = B1l + NQ * KP1;
  float* B2l = B2h + NJ * KP2;
  float* sU = B2l + NJ * KP2;  // [NV][Q][TC]
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;

  const int lane = threadIdx.x & 31, v = threadIdx.x >> 5;  // warp <-> variable
  const int nc = a.m.ncells, nf = a.m.nfaces;
  const int c = blockIdx.x * TC + lane;
  const bool valid = c < nc;
  const int row = v * TC + lane;

  for (int i = threadIdx.x; i < T::B_FLOATS; i += 128) Bs[i] = __ldg(a.tcB + i);
  float w[N];
#pragma unroll
  for (int l = 0; l < N; ++l)
    w[l] = valid ? a.U[(size_t)(v * N + l) * nc + c] : ((v == 0 && l == 0) ? 1.0f : 0.0f);
#pragma unroll
  for (int l = 0; l < KP1; ++l) {
    float hi, lo;
    tc_split(l < N ? w[l] : 0.0f, hi, lo);
    A1h[tc_off(row, l, KP1)] = hi;
    A1l[tc_off(row, l, KP1)] = lo;
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (v == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem(&tmem_base)),
                 "r"(T::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  // MMA 1: nodal values at the volume points
  if (threadIdx.x == 0) {
    tc_gemm_split<KP1, NQ, M>(tmem, A1h, A1l, B1h, B1l);
    tc_commit(&mbar[0]);
  }
  bool ok = tc_wait(&mbar[0], 0);
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t trow = (uint32_t)(v * 32) << 16;
  {
    float u[16];
    tc_ld16(tmem + trow, u);
#pragma unroll
    for (int q = 0; q < Q; ++q) sU[(v * Q + q) * TC + lane] = u[q];
  }
  __syncthreads();

  // Euler fluxes at the points of this thread -> volume part of A2
  const float g1 = (float)a.gamma - 1.0f;
  for (int q = v; q < Q; q += NV) {
    float u[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) u[vv] = sU[(vv * Q + q) * TC + lane];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      float f[NV];
      euler_flux<float, 2>(u, d, g1, f);
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) {
        float hi, lo;
        tc_split(f[vv], hi, lo);
        A2h[tc_off(vv * TC + lane, d * Q + q, KP2)] = hi;
        A2l[tc_off(vv * TC + lane, d * Q + q, KP2)] = lo;
      }
    }
  }
  // face fluxes of this variable -> surface part of A2 (zero beyond)
#pragma unroll
  for (int sd = 0; sd < 4; ++sd) {
    const int e = valid ? a.m.sface[(size_t)sd * nc + c] : 0;
#pragma unroll
    for (int q = 0; q < QF; ++q) {
      const float x = valid ? a.F[((size_t)v * QF + q) * nf + e] : 0.0f;
      float hi, lo;
      tc_split(x, hi, lo);
      A2h[tc_off(row, T::KV + sd * QF + q, KP2)] = hi;
      A2l[tc_off(row, T::KV + sd * QF + q, KP2)] = lo;
    }
  }
#pragma unroll
  for (int k = T::KV + T::KS; k < KP2; ++k) {
    A2h[tc_off(row, k, KP2)] = 0.0f;
    A2l[tc_off(row, k, KP2)] = 0.0f;
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  // MMA 2: volume minus surface integrals
  if (threadIdx.x == 0) {
    tc_gemm_split<KP2, NJ, M>(tmem + NQ, A2h, A2l, B2h, B2l);
    tc_commit(&mbar[1]);
  }
  ok = tc_wait(&mbar[1], 0) && ok;
  asm volatile("tcgen05.fence::after_thread_sync;");
  float acc[16];
  tc_ld16(tmem + trow + NQ, acc);
  if (!ok && lane == 0) atomicOr(a.status, 1 << DG_ERR_TIMEOUT_BIT);

  if (valid && ok) {
    const float pre = a.pre[a.m.level[c]];
    const float dtv = a.dt ? (float)a.dt[cell_problem(a.m, c)] : 1.0f;
    const float pv = a.pre_prob ? a.pre_prob[cell_problem(a.m, c)] : pre;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float rhs = pv * acc[j];
      const size_t idx = (size_t)(v * N + j) * nc + c;
      for (int oo = 0; oo < a.n_out; ++oo) {
        float val = a.ck[oo] * dtv * rhs;
        for (int r = 0; r < a.n_in; ++r) {
          const float cr = a.C[oo][r];
          if (cr == 0.0f) continue;
          val += cr * ((a.in[r] == a.U) ? w[j] : a.in[r][idx]);
        }
        a.out[oo][idx] = val;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (v == 0)
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
        B2h[tc_off(j, d * S::Q + q, T::KP2)] = hi;
        B2l[tc_off(j, d * S::Q + q, T::KP2)] = lo;
      }
    for (int sd = 0; sd < 4; ++sd)
      for (int q = 0; q < S::QF; ++q) {
        const double sc = (sd & 1) ? 1.0 : -1.0;  // outward normal sign of the side
        float hi, lo;
        split(-sc * Tab[S::OFF_PHIFW + ((sd * S::NVAR + 0) * S::QF + q) * S::N + j], hi, lo);
        B2h[tc_off(j, T::KV + sd * S::QF + q, T::KP2)] = hi;
        B2l[tc_off(j, T::KV + sd * S::QF + q, T::KP2)] = lo;
      }
  }
}

template <int K>
cudaError_t launch_cell_tc(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const StageArgs<float>*>(pa);
  using T = TcShape<K>;
  if (a.m.ncells == 0) return cudaSuccess;
  cell_update_tc_kernel<K><<<(a.m.ncells + T::TC - 1) / T::TC, 128, T::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int K>
cudaError_t prepare_cell_tc() {
  return cudaFuncSetAttribute(cell_update_tc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TcShape<K>::SMEM);
}

}  // namespace dgi
