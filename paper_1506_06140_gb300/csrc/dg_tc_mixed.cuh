// Tensor-core cell kernel for the mixed precision mode: FP64 state, FP32
// right-hand side in perturbation form (see dg_mixed.cuh), with the two
// contractions of the cell update on the tensor cores exactly as in
// cell_update_tc_kernel (split-TF32 operands, FP32 accumulation in TMEM):
//   MMA 1: perturbation weights (l >= 1) -> perturbations at the Gauss points;
//   MMA 2: [flux perturbations | face fluxes G (+ D)] -> volume - surface terms.
// The cell mean enters only as each cell's reference state.
#pragma once
#include "dg_mixed.cuh"
#include "dg_tc.cuh"

namespace dgi {

template <int K>
__global__ void __launch_bounds__(256, 3) cell_update_tc_mixed_kernel(const MixedArgs x) {
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
  const StageArgs<double>& a = x.a;
  extern __shared__ __align__(1024) float sm[];
  float* A1h = sm;
  float* A1l = A1h + M * KP1;
  float* sU = sm;  // [NV][Q][TC] perturbations, over A1 once MMA 1 has read it
  float* A2h = sm + T::A1_FLOATS;
  float* A2l = A2h + M * KP2;
  float* B1h = A2l + M * KP2;
  float* B1l = B1h + NQ * KP1;
  float* B2h = B1l + NQ * KP1;
  float* B2l = B2h + NJ * KP2;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ float sRef[NV * TC], sRes[NV * TC];  // reference state and residual per (var, cell)

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int v = warp & 3, half = warp >> 2;
  const int nc = a.m.ncells, nf = a.m.nfaces;
  const int ntiles = (nc + TC - 1) / TC;
  const int row = v * TC + lane;

  for (int i = threadIdx.x; i < T::B_FLOATS; i += 256) B1h[i] = __ldg(x.tcB + i);
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

  // this thread's share of a tile's inputs, loaded a tile ahead: perturbation
  // weights l = half*WH + i of (v, c), the mean's reference and residual
  // (half 0, which holds l = 0), and G (+ D on minus sides) of sides 2*half, 2*half+1
  float wn[WH], xn[2][QF], ubn = 0.0f, resn = 0.0f;
  auto load_tile = [&](int t) {
    const int cc = t * TC + lane;
    const bool in = t < ntiles && cc < nc;
    const size_t i0 = (size_t)v * N * nc + cc;
#pragma unroll
    for (int i = 0; i < WH; ++i) {
      const int l = half * WH + i;
      wn[i] = 0.0f;
      if (!in || l >= N) continue;
      if (l == 0) {
        float hi, lo;
        if (x.wf_mode == 2) {
          hi = x.Wf[i0];
          lo = x.Wlo[(size_t)v * nc + cc];
        } else {
          df_split(a.U[i0], hi, lo);
          if (x.wf_mode == 1) {
            x.Wf[i0] = hi;
            x.Wlo[(size_t)v * nc + cc] = lo;
          }
        }
        mixed_mean_split(hi, lo, x.R, i0, ubn, resn);
      } else {
        const size_t il = i0 + (size_t)l * nc;
        float wl;
        if (x.wf_mode == 2) {
          wl = x.Wf[il];
        } else {
          wl = f32_round(a.U[il]);
          if (x.wf_mode == 1) x.Wf[il] = wl;
        }
        wn[i] = x.R ? wl + x.R[il] : wl;
      }
    }
    if (!in) {  // padding cells: unit density at rest, no perturbation
      ubn = v == 0 ? 1.0f : 0.0f;
      resn = 0.0f;
    }
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int sd = 2 * half + s2;
      const int e = in ? a.m.sface[(size_t)sd * nc + cc] : 0;
      const float dv = (in && !(sd & 1)) ? x.D[(size_t)v * nf + e] : 0.0f;
#pragma unroll
      for (int q = 0; q < QF; ++q) xn[s2][q] = in ? x.G[((size_t)v * QF + q) * nf + e] + dv : 0.0f;
    }
  };
  load_tile(blockIdx.x);

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, phase ^= 1u) {
    const int c = tile * TC + lane;
    const bool valid = c < nc;
    if (half == 0) {
      sRef[v * TC + lane] = ubn;
      sRes[v * TC + lane] = resn;
    }
    // perturbation weights -> A1
#pragma unroll
    for (int g = 0; g < G1H; ++g)
      if ((half * G1H + g) * 4 < KP1) tc_put4(A1h, A1l, tc_off(row, (half * G1H + g) * 4, KP1), &wn[4 * g]);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_gemm_split<KP1, NQ, M>(tmem, A1h, A1l, B1h, B1l);
      tc_commit(&mbar[0]);
    }
    // while MMA 1 runs: face fluxes of two sides -> surface part of A2
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      float xf[QFP];
#pragma unroll
      for (int q = 0; q < QFP; ++q) xf[q] = q < QF ? xn[s2][q] : 0.0f;
#pragma unroll
      for (int g = 0; g < QFP / 4; ++g)
        tc_put4(A2h, A2l, tc_off(row, T::KV + (2 * half + s2) * QFP + 4 * g, KP2), &xf[4 * g]);
    }
    load_tile(tile + gridDim.x);
    // while MMA 1 runs: delta-register combination of the inputs (FP32)
    float base[JH];
#pragma unroll
    for (int jj = 0; jj < JH; ++jj) base[jj] = 0.0f;
    if (x.delta && valid) {
      for (int r = 0; r < x.n_inR; ++r) {
        const float cr = x.Cf[r];
#pragma unroll
        for (int jj = 0; jj < JH; ++jj) {
          const int j = half * JH + jj;
          if (j < N) base[jj] += cr * x.inR[r][(size_t)(v * N + j) * nc + c];
        }
      }
    }
    ok = tc_wait(&mbar[0], phase) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;");
    {
      float u[16];
      tc_ld16(tmem + trow, u);
      const float res = sRes[v * TC + lane];
      // this thread saw MMA 1 complete, so its reads of A1 are over: sU may overwrite A1
#pragma unroll
      for (int i = 0; i < QH; ++i) {
        const int q = half * QH + i;
        const float val = half ? (QH + i < 16 ? u[QH + i] : 0.0f) : u[i];
        if (q < Q) sU[(v * Q + q) * TC + lane] = val + res;
      }
    }
    __syncthreads();
    // flux perturbations in direction d at points 4g..4g+3 (task = warp) -> volume part of A2
    if (warp < 2 * NG) {
      const int d = warp & 1, g = warp >> 1;
      float ub[NV];
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) ub[vv] = sRef[vv * TC + lane];
      const RefState<float, 2> rs = ref_state<float, 2>(ub, g1);
      float f[NV][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int q = 4 * g + i;
        float du[NV], fd[NV];
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) du[vv] = q < Q ? sU[(vv * Q + q) * TC + lane] : 0.0f;
        const Pert<float, 2> pq = perturb<float, 2>(rs, du, g1);
        if (d == 0)
          euler_dflux<float, 2>(rs, du, pq, 0, fd);
        else
          euler_dflux<float, 2>(rs, du, pq, 1, fd);
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) f[vv][i] = q < Q ? fd[vv] : 0.0f;
      }
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) tc_put4(A2h, A2l, tc_off(vv * TC + lane, d * QP + 4 * g, KP2), f[vv]);
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
      const int pb = cell_problem(a.m, c);
      const double pre = a.pre_prob ? a.pre_prob[pb] : a.pre[a.m.level[c]];
      const double dtv = a.dt ? a.dt[pb] : 1.0;
      if (x.delta) {
        const float sc = x.ckf * f32_round(dtv * pre);
#pragma unroll
        for (int jj = 0; jj < JH; ++jj) {
          const int j = half * JH + jj;
          const float rhs = half ? (JH + jj < 16 ? acc[JH + jj] : 0.0f) : acc[jj];
          if (j >= N) continue;
          const size_t idx = (size_t)(v * N + j) * nc + c;
          const float val = base[jj] + sc * rhs;
          if (x.outR) x.outR[idx] = val;
          else a.out[0][idx] = a.U[idx] + f64_exact(val);
        }
      } else {
#pragma unroll
        for (int jj = 0; jj < JH; ++jj) {
          const int j = half * JH + jj;
          const float rhs32 = half ? (JH + jj < 16 ? acc[JH + jj] : 0.0f) : acc[jj];
          if (j >= N) continue;
          const size_t idx = (size_t)(v * N + j) * nc + c;
          const double rhs = pre * f64_exact(rhs32);
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

template <int K>
struct TcMixedGrid {
  static inline int ctas = 0;  // resident CTAs on the whole device (set by prepare_cell_tc_mixed)
};

template <int K>
cudaError_t launch_cell_tc_mixed(const void* px, cudaStream_t s) {
  const auto& x = *static_cast<const MixedArgs*>(px);
  using T = TcShape<K>;
  if (x.a.m.ncells == 0) return cudaSuccess;
  const int ntiles = (x.a.m.ncells + T::TC - 1) / T::TC;
  const int grid = TcMixedGrid<K>::ctas > 0 && TcMixedGrid<K>::ctas < ntiles ? TcMixedGrid<K>::ctas : ntiles;
  cell_update_tc_mixed_kernel<K><<<grid, 256, T::SMEM, s>>>(x);
  return cudaGetLastError();
}

template <int K>
cudaError_t prepare_cell_tc_mixed() {
  cudaError_t e = cudaFuncSetAttribute(cell_update_tc_mixed_kernel<K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcShape<K>::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(cell_update_tc_mixed_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
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
  if ((e = cudaFuncGetAttributes(&fa, cell_update_tc_mixed_kernel<K>)) != cudaSuccess) return e;
  const int by_smem = smem_sm / (int)(TcShape<K>::SMEM + fa.sharedSizeBytes + smem_rsv);
  const int by_regs = regs_sm / ((fa.numRegs > 0 ? fa.numRegs : 1) * 256);
  int per_sm = by_smem < by_regs ? by_smem : by_regs;
  if (per_sm > 8) per_sm = 8;  // 2048 threads per SM
  TcMixedGrid<K>::ctas = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

}  // namespace dgi
