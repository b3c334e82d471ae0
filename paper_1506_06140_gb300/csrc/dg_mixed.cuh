// The two kernels of one RK stage (paper Sec. 2.4, eqs. dg_term2, dg_term3,
// spatial_discretisation) for an FP64 state whose right-hand side is
// evaluated in FP32 in perturbation form.
//
// Every cell c has a reference state ubar_c = its weight w_0 (phi_0 = 1),
// rounded to FP32.  Because the volume integral of a constant flux against
// the basis gradients equals its surface integral (both Gauss rules are
// exact for these polynomial degrees, also on the halves or quarters of a
// hanging face), the cell's right-hand side is unchanged when f(ubar_c) is
// subtracted from the point fluxes and from the face fluxes it integrates.
// The kernels therefore carry only perturbations through FP32:
//   * the point states are ubar_c + du with du from the weights l >= 1 plus
//     the FP64 rounding residual of ubar_c;
//   * the point fluxes are f(ubar_c + du) - f(ubar_c) (euler_dflux);
//   * each face stores G = F*(uL, uR) - f(ubar_m) relative to its minus cell
//     m (the existing cell at a domain boundary) and D = f(ubar_m) - f(ubar_p);
//     the minus cell integrates G and the plus cell G + D.
// Rounding errors then scale with the variation of the solution across a
// cell and its neighbours instead of with the size of the fluxes, which is
// what keeps an FP32 right-hand side usable on fine meshes.  The stage
// combination and the state stay in FP64.
#pragma once
#include <cuda_runtime.h>

#include "dg_convert.cuh"
#include "dg_internal.h"
#include "dg_physics.cuh"
#include "dg_stage.cuh"

namespace dgi {

// d = hi + lo with hi = d truncated to FP32 and lo the remaining 29 mantissa bits,
// rounded to FP32 (|d - hi - lo| <= 2^-47 |d|); integer instructions and one
// integer-to-float conversion.  |d| below 2^-126 gives 0 + 0.
__device__ __forceinline__ void df_split(double d, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned e = (h32 >> 20) & 0x7FFu;
  hi = e > 896u ? __uint_as_float((h32 & 0x80000000u) | ((e - 896u) << 23) | ((h32 & 0xFFFFFu) << 3) |
                                  (l32 >> 29))
                : 0.0f;
  // the dropped bits are worth r 2^(e - 1075); that power of two as an FP32
  const float scale = e > 948u ? __uint_as_float((e - 948u) << 23) : 0.0f;
  const float rl = __uint2float_rn(l32 & 0x1FFFFFFFu) * scale;
  lo = __uint_as_float(__float_as_uint(rl) | (h32 & 0x80000000u));
}

// exact sum s + err = a + b (Knuth's TwoSum)
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
  return s;
}

// mean (weight 0) of one variable of a cell as reference + residual: the
// state is W (+ R, the FP32 delta of a stage register, when R is given)
__device__ __forceinline__ void mixed_mean_split(float hi, float lo, const float* R, size_t idx,
                                                 float& ub, float& res) {
  if (R) {
    float e;
    ub = two_sum(hi, R[idx], e);
    res = lo + e;
  } else {
    ub = hi;
    res = lo;
  }
}

__device__ __forceinline__ void mixed_mean(double w0, const float* R, size_t idx, float& ub,
                                           float& res) {
  float hi, lo;
  df_split(w0, hi, lo);
  mixed_mean_split(hi, lo, R, idx, ub, res);
}

// FP32 weights l >= 1 of one variable of a cell (W, or W + R) and its mean
// as reference + residual: from the FP64 state, or (wf_mode 2) from the FP32
// split of W that the step's first cell kernel wrote
template <int N>
__device__ __forceinline__ void mixed_weights(const MixedArgs& x, size_t i0, int v, int c, size_t nc,
                                              float* w, float& ub, float& res) {
  if (x.wf_mode == 2) {
    mixed_mean_split(x.Wf[i0], x.Wlo[(size_t)v * nc + c], x.R, i0, ub, res);
#pragma unroll
    for (int l = 1; l < N; ++l) w[l] = x.Wf[i0 + (size_t)l * nc];
  } else {
    const double* Wc = x.a.U + i0;
    mixed_mean(Wc[0], x.R, i0, ub, res);
#pragma unroll
    for (int l = 1; l < N; ++l) w[l] = f32_round(Wc[(size_t)l * nc]);
  }
  if (x.R) {
#pragma unroll
    for (int l = 1; l < N; ++l) w[l] += x.R[i0 + (size_t)l * nc];
  }
}

// FP32 trace of the weights l >= 1 of one variable of a cell on side s, plus
// the residual ubar - fl32(ubar) (the trace of phi_0 is 1 at every point)
template <int DIM, int K, int DIR>
__device__ __forceinline__ void mixed_trace(const MixedArgs& x, int cell, int s, int var, int v,
                                            float& ubar, float& res, float* du) {
  using S = Shape<DIM, K>;
  const int nc = x.a.m.ncells;
  const size_t i0 = (size_t)v * S::N * nc + cell;
  float w[S::N];
  mixed_weights<S::N>(x, i0, v, cell, nc, w, ubar, res);
  w[0] = 0.0f;
  if (var == 0) {
    face_trace<float, DIM, K, DIR>(x.t, w, s, x.t.P, x.t.P, du);
  } else {
    const int h0 = (var - 1) & 1, h1 = ((var - 1) >> 1) & 1;
    face_trace<float, DIM, K, DIR>(x.t, w, s, x.t.PH[h0], x.t.PH[h1], du);
  }
}

template <int DIM, int K>
struct MixedFaceTile {
  using S = Shape<DIM, K>;
  static constexpr int FB = 32;  // default faces per block; kernels for 16, 32, 64
  static constexpr int FB_MAX = 64;
  // reference [NV][FB], reference difference [NV][FB], perturbations [2][NV][QF][FB]
  static constexpr size_t smem(int fb) { return (size_t)(2 * S::NV + 2 * S::NV * S::QF) * fb * sizeof(float); }
};

template <int DIM, int K, int FB>
__global__ void __launch_bounds__(FB * Shape<DIM, K>::NV)
    face_flux_mixed_kernel(const MixedArgs x) {
  pdl_wait();
  using S = Shape<DIM, K>;
  constexpr int NV = S::NV, QF = S::QF, THREADS = FB * NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sRef = reinterpret_cast<float*>(smem_raw);  // [NV][FB]
  float* sDel = sRef + NV * FB;                       // [NV][FB]
  float* sP = sDel + NV * FB;                         // [2][NV][QF][FB]
  const StageArgs<double>& a = x.a;
  const int nf = a.m.nfaces;
  const int fl = threadIdx.x % FB, v = threadIdx.x / FB;
  const int f = blockIdx.x * FB + fl;
  if (f < nf) {
    const unsigned info = a.m.finfo[f];
    const int dir = info & 3;
    const int vm = (info >> 2) & 7, vp = (info >> 5) & 7;
    const int cm = a.m.fm[f], cp = a.m.fp[f];
    float dm[QF], dp[QF], bm = 0.0f, bp = 0.0f, rm = 0.0f, rp = 0.0f;
    // the minus cell sees the face as its + side (s = 1), the plus cell as its - side
    auto trace = [&](int cell, int s, int var, float& ub, float& res, float* du) {
      if (dir == 0) mixed_trace<DIM, K, 0>(x, cell, s, var, v, ub, res, du);
      else if (dir == 1) mixed_trace<DIM, K, 1>(x, cell, s, var, v, ub, res, du);
      else if constexpr (DIM == 3) mixed_trace<DIM, K, DIM - 1>(x, cell, s, var, v, ub, res, du);
    };
    if (cm >= 0) trace(cm, 1, vm, bm, rm, dm);
    if (cp >= 0) trace(cp, 0, vp, bp, rp, dp);
    // reference: the minus cell's (the plus cell's at a minus-side boundary);
    // om, op: offsets of the two sides' states from it
    float ref, del = 0.0f, om, op;
    if (cm >= 0) {
      ref = bm;
      om = rm;
      if (cp >= 0) {
        del = bp - bm;
        op = del + rp;
      } else {
        op = om;
#pragma unroll
        for (int q = 0; q < QF; ++q) dp[q] = dm[q];
      }
    } else {
      ref = bp;
      op = rp;
      om = op;
#pragma unroll
      for (int q = 0; q < QF; ++q) dm[q] = dp[q];
    }
    sRef[v * FB + fl] = ref;
    sDel[v * FB + fl] = del;
#pragma unroll
    for (int q = 0; q < QF; ++q) {
      sP[((0 * NV + v) * QF + q) * FB + fl] = dm[q] + om;
      sP[((1 * NV + v) * QF + q) * FB + fl] = dp[q] + op;
    }
  }
  __syncthreads();
  const float gamma = x.gamf, g1 = x.g1f;
  // HLLC in perturbation form at every (face, point) of the block
  for (int item = threadIdx.x; item < FB * QF; item += THREADS) {
    const int ff = item % FB, q = item / FB;
    const int f2 = blockIdx.x * FB + ff;
    if (f2 >= nf) continue;
    const int d2 = a.m.finfo[f2] & 3;
    float ub[NV], dL[NV], dR[NV], G[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      ub[vv] = sRef[vv * FB + ff];
      dL[vv] = sP[((0 * NV + vv) * QF + q) * FB + ff];
      dR[vv] = sP[((1 * NV + vv) * QF + q) * FB + ff];
    }
    const RefState<float, DIM> r = ref_state<float, DIM>(ub, g1);
    if (d2 == 0) hllc_dflux<float, DIM>(r, dL, dR, 0, gamma, G);
    else if (d2 == 1) hllc_dflux<float, DIM>(r, dL, dR, 1, gamma, G);
    else hllc_dflux<float, DIM>(r, dL, dR, DIM - 1, gamma, G);
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) x.G[((size_t)vv * QF + q) * nf + f2] = G[vv];
  }
  // D = f(ubar_m) - f(ubar_p) = -(f(ubar_m + del) - f(ubar_m)) per face
  for (int ff = threadIdx.x; ff < FB; ff += THREADS) {
    const int f2 = blockIdx.x * FB + ff;
    if (f2 >= nf) continue;
    const int d2 = a.m.finfo[f2] & 3;
    float ub[NV], del[NV], df[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      ub[vv] = sRef[vv * FB + ff];
      del[vv] = sDel[vv * FB + ff];
    }
    const RefState<float, DIM> r = ref_state<float, DIM>(ub, g1);
    const Pert<float, DIM> pq = perturb<float, DIM>(r, del, g1);
    if (d2 == 0) euler_dflux<float, DIM>(r, del, pq, 0, df);
    else if (d2 == 1) euler_dflux<float, DIM>(r, del, pq, 1, df);
    else euler_dflux<float, DIM>(r, del, pq, DIM - 1, df);
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) x.D[(size_t)vv * nf + f2] = -df[vv];
  }
}

template <int DIM, int K>
struct MixedCellTile {
  using S = Shape<DIM, K>;
  static constexpr size_t PER_CELL =
      (size_t)(S::NV + S::NV * S::Q + DIM * S::NV * S::Q) * sizeof(float);
  static constexpr int TC = PER_CELL * 32 > 96 * 1024 ? 16 : 32;  // default cells per block
  static constexpr int TC_MAX = PER_CELL * 64 <= 200 * 1024 ? 64 : (PER_CELL * 32 <= 200 * 1024 ? 32 : 16);
  static constexpr size_t smem(int tc) { return PER_CELL * tc; }
};

// surface integral of one side from G (+ D on the plus side of each face)
template <int DIM, int K, int SD>
__device__ __forceinline__ void surface_from_faces_mixed(const MixedArgs& x, int c, int v,
                                                         unsigned coarse, float* acc) {
  using S = Shape<DIM, K>;
  constexpr int DIR = SD >> 1, SS = SD & 1;
  const int nc = x.a.m.ncells, nf = x.a.m.nfaces;
  const int e0 = x.a.m.sface[(size_t)SD * nc + c];
  float fq[S::QF];
  if (!((coarse >> SD) & 1)) {
    const float dv = SS ? 0.0f : x.D[(size_t)v * nf + e0];
#pragma unroll
    for (int q = 0; q < S::QF; ++q) fq[q] = x.G[((size_t)v * S::QF + q) * nf + e0] + dv;
    surface_side<float, DIM, K, DIR, SS>(x.t, x.t.PW, x.t.PW, fq, 1.0f, acc);
  } else {
    const float sub = 1.0f / (float)S::NSUB;
#pragma unroll
    for (int h = 0; h < S::NSUB; ++h) {
      const float dv = SS ? 0.0f : x.D[(size_t)v * nf + e0 + h];
#pragma unroll
      for (int q = 0; q < S::QF; ++q) fq[q] = x.G[((size_t)v * S::QF + q) * nf + e0 + h] + dv;
      surface_side<float, DIM, K, DIR, SS>(x.t, x.t.PWH[h & 1], x.t.PWH[(h >> 1) & 1], fq, sub, acc);
    }
  }
}

template <int DIM, int K, int TC>
__global__ void __launch_bounds__(TC * Shape<DIM, K>::NV)
    cell_update_mixed_kernel(const MixedArgs x) {
  pdl_wait();
  using S = Shape<DIM, K>;
  constexpr int NV = S::NV, Q = S::Q, N = S::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sRef = reinterpret_cast<float*>(smem_raw);  // [NV][TC]
  float* sU = sRef + NV * TC;                         // [NV][Q][TC] perturbations
  float* sF = sU + NV * Q * TC;                       // [DIM][NV][Q][TC] flux perturbations
  const StageArgs<double>& a = x.a;
  const int tc = threadIdx.x % TC, v = threadIdx.x / TC;
  const int nc = a.m.ncells;
  const int c = blockIdx.x * TC + tc;
  const bool valid = c < nc;

  // 1. reference and perturbation of this variable at the points
  {
    const size_t i0 = (size_t)v * N * nc + c;
    float ub = v == 0 ? 1.0f : 0.0f, res = 0.0f;  // padding cells: unit density at rest
    float w[N], u[Q];
    w[0] = 0.0f;
#pragma unroll
    for (int l = 1; l < N; ++l) w[l] = 0.0f;
    if (valid) {
      if (x.wf_mode == 1) {
        // first stage of a step: keep the FP32 split of W for the later stages
        float hi, lo;
        df_split(a.U[i0], hi, lo);
        x.Wf[i0] = hi;
        x.Wlo[(size_t)v * nc + c] = lo;
#pragma unroll
        for (int l = 1; l < N; ++l) x.Wf[i0 + (size_t)l * nc] = f32_round(a.U[i0 + (size_t)l * nc]);
      }
      mixed_weights<N>(x, i0, v, c, nc, w, ub, res);
      w[0] = 0.0f;
    }
    modal_to_nodal<float, DIM, K>(x.t, w, u);
    sRef[v * TC + tc] = ub;
#pragma unroll
    for (int q = 0; q < Q; ++q) sU[(v * Q + q) * TC + tc] = u[q] + res;
  }
  __syncthreads();

  // 2. flux perturbations at the points of this thread
  const float g1 = x.g1f;
  {
    float ub[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) ub[vv] = sRef[vv * TC + tc];
    const RefState<float, DIM> r = ref_state<float, DIM>(ub, g1);
    for (int q = v; q < Q; q += NV) {
      float du[NV];
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) du[vv] = sU[(vv * Q + q) * TC + tc];
      const Pert<float, DIM> pq = perturb<float, DIM>(r, du, g1);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        float f[NV];
        euler_dflux<float, DIM>(r, du, pq, d, f);
#pragma unroll
        for (int vv = 0; vv < NV; ++vv) sF[((d * NV + vv) * Q + q) * TC + tc] = f[vv];
      }
    }
  }
  __syncthreads();
  if (!valid) return;

  // 3. volume and surface integrals of this variable (FP32)
  float acc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l] = 0.0f;
  {
    float f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = sF[((0 * NV + v) * Q + q) * TC + tc];
    volume_dir<float, DIM, K, 0>(x.t, f, acc);
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = sF[((1 * NV + v) * Q + q) * TC + tc];
    volume_dir<float, DIM, K, 1>(x.t, f, acc);
    if constexpr (DIM == 3) {
#pragma unroll
      for (int q = 0; q < Q; ++q) f[q] = sF[((2 * NV + v) * Q + q) * TC + tc];
      volume_dir<float, DIM, K, DIM - 1>(x.t, f, acc);
    }
  }
  const unsigned coarse = a.m.scoarse[c];
  surface_from_faces_mixed<DIM, K, 0>(x, c, v, coarse, acc);
  surface_from_faces_mixed<DIM, K, 1>(x, c, v, coarse, acc);
  surface_from_faces_mixed<DIM, K, 2>(x, c, v, coarse, acc);
  surface_from_faces_mixed<DIM, K, 3>(x, c, v, coarse, acc);
  if constexpr (DIM == 3) {
    surface_from_faces_mixed<DIM, K, 2 * DIM - 2>(x, c, v, coarse, acc);
    surface_from_faces_mixed<DIM, K, 2 * DIM - 1>(x, c, v, coarse, acc);
  }

  // 4. epilogue
  const int pb = cell_problem(a.m, c);
  const double pre = a.pre_prob ? a.pre_prob[pb] : a.pre[a.m.level[c]];
  const double dtv = a.dt ? a.dt[pb] : 1.0;
  const size_t i0 = (size_t)(v * N) * nc + c;
  if (x.delta) {
    // delta registers: R_out = sum_r C_r R_r + ck dt dW/dt in FP32 (the
    // coefficients of a stage state sum to one, so W drops out); the last
    // stage adds that increment to W in FP64.  The terms are added in that
    // order; the loop over the inputs runs outside the coefficient loop.
    const float sc = x.ckf * f32_round(dtv * pre);
    float val[N];
#pragma unroll
    for (int j = 0; j < N; ++j) val[j] = sc * acc[j];
#pragma unroll
    for (int r = 0; r < MAX_IN; ++r) {
      if (r >= x.n_inR) break;
      const float cr = x.Cf[r];
      const float* src = x.inR[r];
#pragma unroll
      for (int j = 0; j < N; ++j) val[j] += cr * src[i0 + (size_t)j * nc];
    }
    if (x.outR) {
#pragma unroll
      for (int j = 0; j < N; ++j) x.outR[i0 + (size_t)j * nc] = val[j];
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j) a.out[0][i0 + (size_t)j * nc] = a.U[i0 + (size_t)j * nc] + f64_exact(val[j]);
    }
    return;
  }
  // FP64 registers: out_o = ck[o] dt pre acc + sum_r C[o][r] in_r, in that order
#pragma unroll
  for (int oo = 0; oo < MAX_OUT; ++oo) {
    if (oo >= a.n_out) break;
    const double ckv = a.ck[oo] * dtv;
    double val[N];
#pragma unroll
    for (int j = 0; j < N; ++j) val[j] = ckv * (pre * f64_exact(acc[j]));
#pragma unroll
    for (int r = 0; r < MAX_IN; ++r) {
      if (r >= a.n_in) break;
      const double cr = a.C[oo][r];
      if (cr == 0.0) continue;
      const double* src = a.in[r];
#pragma unroll
      for (int j = 0; j < N; ++j) val[j] += cr * src[i0 + (size_t)j * nc];
    }
#pragma unroll
    for (int j = 0; j < N; ++j) a.out[oo][i0 + (size_t)j * nc] = val[j];
  }
}

template <int DIM, int K>
cudaError_t launch_face_mixed(const void* px, cudaStream_t s) {
  const auto& x = *static_cast<const MixedArgs*>(px);
  using FT = MixedFaceTile<DIM, K>;
  constexpr int NV = Shape<DIM, K>::NV;
  if (x.a.m.nfaces == 0) return cudaSuccess;
  const int fb = x.a.face_tile == 16 || x.a.face_tile == 64 ? x.a.face_tile : 32;
  const int grid = (x.a.m.nfaces + fb - 1) / fb;
  const bool pdl = x.a.pdl != 0;
  if (fb == 16) return launch_pdl(pdl, face_flux_mixed_kernel<DIM, K, 16>, grid, 16 * NV, FT::smem(16), s, x);
  if (fb == 64) return launch_pdl(pdl, face_flux_mixed_kernel<DIM, K, 64>, grid, 64 * NV, FT::smem(64), s, x);
  return launch_pdl(pdl, face_flux_mixed_kernel<DIM, K, 32>, grid, 32 * NV, FT::smem(32), s, x);
}

template <int DIM, int K>
cudaError_t launch_cell_mixed(const void* px, cudaStream_t s) {
  const auto& x = *static_cast<const MixedArgs*>(px);
  using CT = MixedCellTile<DIM, K>;
  constexpr int NV = Shape<DIM, K>::NV;
  if (x.a.m.ncells == 0) return cudaSuccess;
  const int tc = (x.a.cell_tile == 16 || x.a.cell_tile == 32 || x.a.cell_tile == 64) && x.a.cell_tile <= CT::TC_MAX
                     ? x.a.cell_tile
                     : CT::TC;
  const int grid = (x.a.m.ncells + tc - 1) / tc;
  if (tc == 16) {
    return launch_pdl(x.a.pdl != 0, cell_update_mixed_kernel<DIM, K, 16>, grid, 16 * NV, CT::smem(16), s, x);
  } else if (tc == 32) {
    if constexpr (CT::TC_MAX >= 32)
      return launch_pdl(x.a.pdl != 0, cell_update_mixed_kernel<DIM, K, 32>, grid, 32 * NV, CT::smem(32), s, x);
  } else {
    if constexpr (CT::TC_MAX >= 64)
      return launch_pdl(x.a.pdl != 0, cell_update_mixed_kernel<DIM, K, 64>, grid, 64 * NV, CT::smem(64), s, x);
  }
  return cudaGetLastError();
}

template <int DIM, int K>
cudaError_t prepare_mixed() {
  using CT = MixedCellTile<DIM, K>;
  using FT = MixedFaceTile<DIM, K>;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(cell_update_mixed_kernel<DIM, K, 16>, attr, (int)CT::smem(16));
  if (e == cudaSuccess && CT::TC_MAX >= 32) {
    if constexpr (CT::TC_MAX >= 32) e = cudaFuncSetAttribute(cell_update_mixed_kernel<DIM, K, 32>, attr, (int)CT::smem(32));
  }
  if (e == cudaSuccess && CT::TC_MAX >= 64) {
    if constexpr (CT::TC_MAX >= 64) e = cudaFuncSetAttribute(cell_update_mixed_kernel<DIM, K, 64>, attr, (int)CT::smem(64));
  }
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(face_flux_mixed_kernel<DIM, K, 16>, attr, (int)FT::smem(16))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(face_flux_mixed_kernel<DIM, K, 32>, attr, (int)FT::smem(32))) != cudaSuccess) return e;
  return cudaFuncSetAttribute(face_flux_mixed_kernel<DIM, K, 64>, attr, (int)FT::smem(64));
}

template <int DIM, int K>
MixedSet make_mixed_set() {
  MixedSet ms;
  ms.cell_tile = MixedCellTile<DIM, K>::TC;
  ms.cell_tile_max = MixedCellTile<DIM, K>::TC_MAX;
  ms.face_tile = MixedFaceTile<DIM, K>::FB;
  ms.face_tile_max = MixedFaceTile<DIM, K>::FB_MAX;
  ms.face = &launch_face_mixed<DIM, K>;
  ms.cell = &launch_cell_mixed<DIM, K>;
  ms.prepare = &prepare_mixed<DIM, K>;
  return ms;
}

}  // namespace dgi
