// FP32 cell kernel with one thread per cell (paper Sec. 2.4, eqs. dg_term2,
// dg_term3, spatial_discretisation): the thread keeps all variables'
// weights and accumulators in registers and streams over the Gauss points,
// so no shared memory and no barriers are needed.  The contractions are the
// direct [N x Q] products (not sum-factorised): more multiply-adds than the
// tiled kernel, but every table entry is a constant-bank operand of an FMA
// (the tables travel by value in the kernel arguments) and the FP32 pipe,
// not the index arithmetic and shared-memory traffic of the tiled kernel,
// sets the pace.
#pragma once
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "dg_internal.h"
#include "dg_physics.cuh"

namespace dgi {

template <int DIM, int K>
struct DirectTab {
  using S = Shape<DIM, K>;
  float phi[S::Q][S::N];                          // phi_l(xi_q)
  float dphiw[DIM][S::Q][S::N];                   // dphi_l/dxi_d(xi_q) w_q
  float face[2 * DIM][S::NVAR][S::QF][S::N];      // -n_s phi_l(face point) w_q (x sub-face weight)
};

template <int DIM, int K>
struct DirectArgs {
  StageArgs<float> a;
  DirectTab<DIM, K> t;
};

constexpr int DIRECT_THREADS = 128;

template <int DIM, int K, bool AMR>
__global__ void __launch_bounds__(DIRECT_THREADS) cell_update_direct_kernel(const DirectArgs<DIM, K> x) {
  using S = Shape<DIM, K>;
  constexpr int NV = S::NV, N = S::N, Q = S::Q, QF = S::QF;
  const StageArgs<float>& a = x.a;
  const DirectTab<DIM, K>& t = x.t;
  const int nc = a.m.ncells, nf = a.m.nfaces;
  const int c = blockIdx.x * DIRECT_THREADS + threadIdx.x;
  if (c >= nc) return;
  float w[NV][N], acc[NV][N];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int l = 0; l < N; ++l) {
      w[v][l] = a.U[(size_t)(v * N + l) * nc + c];
      acc[v][l] = 0.0f;
    }
  const float g1 = a.gm1;
  // volume: at each point, the state, the fluxes of all directions, and their
  // products with the weighted basis gradients
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float s = 0.0f;
#pragma unroll
      for (int l = 0; l < N; ++l) s += w[v][l] * t.phi[q][l];
      u[v] = s;
    }
    float f[DIM][NV];
    euler_flux_all<float, DIM>(u, g1, f);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int l = 0; l < N; ++l) acc[v][l] += f[d][v] * t.dphiw[d][q][l];
  }
  // surface: the stored face fluxes of each side (NSUB sub-faces on the
  // coarse side of a hanging face, only on refined meshes)
  const unsigned coarse = AMR ? a.m.scoarse[c] : 0u;
#pragma unroll
  for (int sd = 0; sd < 2 * DIM; ++sd) {
    const int e0 = a.m.sface[(size_t)sd * nc + c];
    if (!AMR || !((coarse >> sd) & 1)) {
#pragma unroll
      for (int q = 0; q < QF; ++q)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float fq = a.F[((size_t)v * QF + q) * nf + e0];
#pragma unroll
          for (int l = 0; l < N; ++l) acc[v][l] += fq * t.face[sd][0][q][l];
        }
    } else {
      if constexpr (AMR) {
#pragma unroll
        for (int h = 0; h < S::NSUB; ++h)
#pragma unroll
          for (int q = 0; q < QF; ++q)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              const float fq = a.F[((size_t)v * QF + q) * nf + e0 + h];
#pragma unroll
              for (int l = 0; l < N; ++l) acc[v][l] += fq * t.face[sd][1 + h][q][l];
            }
      }
    }
  }
  // epilogue: out_o = sum_r C[o][r] in_r + ck[o] dt pre dW/dt
  const int pb = cell_problem(a.m, c);
  const float pre = a.pre_prob ? a.pre_prob[pb] : a.pre[a.m.level[c]];
  const float sc = pre * (a.dt ? (float)a.dt[pb] : 1.0f);
  for (int oo = 0; oo < a.n_out; ++oo) {
    const float ck = a.ck[oo] * sc;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const size_t idx = (size_t)(v * N + l) * nc + c;
        float val = ck * acc[v][l];
        for (int r = 0; r < a.n_in; ++r) {
          const float cr = a.C[oo][r];
          if (cr != 0.0f) val += cr * ((a.in[r] == a.U) ? w[v][l] : a.in[r][idx]);
        }
        a.out[oo][idx] = val;
      }
  }
}

// host: the tables from the FP64 scheme tables
template <int DIM, int K>
void fill_direct_tables(const std::vector<double>& Tab, std::vector<unsigned char>& out) {
  using S = Shape<DIM, K>;
  DirectTab<DIM, K> t;
  for (int q = 0; q < S::Q; ++q)
    for (int l = 0; l < S::N; ++l) {
      t.phi[q][l] = (float)Tab[S::OFF_PHI + q * S::N + l];
      for (int d = 0; d < DIM; ++d) t.dphiw[d][q][l] = (float)Tab[S::OFF_DPHIW + (d * S::Q + q) * S::N + l];
    }
  for (int sd = 0; sd < 2 * DIM; ++sd) {
    const double sgn = (sd & 1) ? -1.0 : 1.0;  // minus the outward normal's sign of the side
    for (int var = 0; var < S::NVAR; ++var)
      for (int q = 0; q < S::QF; ++q)
        for (int l = 0; l < S::N; ++l)
          t.face[sd][var][q][l] = (float)(sgn * Tab[S::OFF_PHIFW + ((sd * S::NVAR + var) * S::QF + q) * S::N + l]);
  }
  out.resize(sizeof(t));
  std::memcpy(out.data(), &t, sizeof(t));
}

template <int DIM, int K>
cudaError_t launch_cell_direct(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const StageArgs<float>*>(pa);
  if (a.m.ncells == 0) return cudaSuccess;
  if (!a.dtab) return cudaErrorInvalidValue;
  DirectArgs<DIM, K> x;
  x.a = a;
  std::memcpy(&x.t, a.dtab, sizeof(x.t));
  const int grid = (a.m.ncells + DIRECT_THREADS - 1) / DIRECT_THREADS;
  if (a.m.nnodes > 0) cell_update_direct_kernel<DIM, K, true><<<grid, DIRECT_THREADS, 0, s>>>(x);
  else cell_update_direct_kernel<DIM, K, false><<<grid, DIRECT_THREADS, 0, s>>>(x);
  return cudaGetLastError();
}

}  // namespace dgi
