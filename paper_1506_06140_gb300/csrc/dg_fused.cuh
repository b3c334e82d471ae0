// One RK stage of a 2D uniform mesh in a single kernel: a cell tile plus
// its face halo (paper Sec. 2.4, eqs. dg_term2, dg_term3).  A block takes a
// tile of 8 x 4 cells and
//   1. loads each cell's weights once, stages its nodal values (as the cell
//      kernel) and its traces on all four sides in shared memory; for sides
//      whose neighbour lies outside the tile it also computes that
//      neighbour's trace (the halo);
//   2. computes the HLLC flux of every face of the tile once -- each cell
//      owns its + sides, and its - sides whose neighbour is outside the tile
//      or absent (a transmissive boundary mirrors the state) -- into shared
//      memory;
//   3. runs the cell update: point fluxes, volume integral, the surface
//      integral from the tile's face fluxes, and the stage combination.
// Against the face kernel + cell kernel pair it reads every weight of the
// tile once instead of once per face side, keeps the face fluxes out of
// global memory and saves a launch per stage; the faces on the tile's edges
// are computed by both tiles (76 faces per 32 cells instead of 64).
//
// Traces, fluxes and integrals come from the functions the two-kernel path
// uses, with the same arguments in the same order; the results agree with it
// to rounding (the compiler may contract a multiply and an add into an FMA
// differently in the two kernels).
#pragma once
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_physics.cuh"
#include "dg_stage.cuh"

namespace dgi {

template <typename real, int K>
struct FusedTile {
  using S = Shape<2, K>;
  static constexpr int TX = 8, TY = 4, TC = TX * TY;  // cells of a tile (x fastest)
  static constexpr int THREADS = TC * S::NV;
  // shared memory (reals): point data [2][NV][Q][TC] (the cell kernel's
  // layout, direction 0 over the nodal values), own traces, halo traces and
  // face fluxes, each [4 sides][NV][QF][TC]; the sides' neighbour slots
  static constexpr int PT = 2 * S::NV * S::Q * TC;
  static constexpr int TR = 4 * S::NV * S::QF * TC;
  static constexpr size_t SMEM = (size_t)(PT + 3 * TR) * sizeof(real) + 4 * TC * sizeof(int);
  static int blocks(int nx, int ny) { return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY); }
};

// trace of one variable on side SIDE (= 2 axis + {0: -, 1: +}) at the Gauss points
template <typename real, int K, int SIDE>
__device__ __forceinline__ void fused_trace(const Tab1D<real>& T, const real* w, real* u) {
  face_trace<real, 2, K, (SIDE >> 1)>(T, w, SIDE & 1, T.P, T.P, u);
}

template <typename real, int K>
__global__ void __launch_bounds__(FusedTile<real, K>::THREADS) stage_fused_kernel(const StageArgs<real> a) {
  using S = Shape<2, K>;
  using FT = FusedTile<real, K>;
  constexpr int NV = S::NV, N = S::N, Q = S::Q, QF = S::QF, TC = FT::TC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sU = reinterpret_cast<real*>(smem_raw);  // [NV][Q][TC]
  real* sFl = sU;                                // [2][NV][Q][TC], direction 0 over sU
  real* sT = sU + FT::PT;                        // own traces [4][NV][QF][TC]
  real* sH = sT + FT::TR;                        // halo traces [4][NV][QF][TC]
  real* sF = sH + FT::TR;                        // fluxes of the owned faces [4][NV][QF][TC]
  int* sSlot = reinterpret_cast<int*>(sF + FT::TR);  // [4][TC]: neighbour's slot, -1 outside, -2 none
  const Tab1D<real>& T = a.t1;
  const int tc = threadIdx.x % TC, v = threadIdx.x / TC;
  const int nx = a.m.n[0], ny = a.m.n[1], nc = a.m.ncells;
  const int tiles_x = (nx + FT::TX - 1) / FT::TX;
  const int x0 = (blockIdx.x % tiles_x) * FT::TX, y0 = (blockIdx.x / tiles_x) * FT::TY;
  const int gx = x0 + tc % FT::TX, gy = y0 + tc / FT::TX;
  const bool valid = gx < nx && gy < ny;
  const int c = valid ? gx + nx * gy : 0;

  // neighbours of this cell: tile slot, -1 (outside the tile), -2 (none)
  int slot[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int nb = valid ? a.m.nbr[(size_t)s * nc + c] : -1;
    slot[s] = -2;
    if (nb >= 0) {
      const int bx = nb % nx, by = nb / nx;
      slot[s] = (bx >= x0 && bx < x0 + FT::TX && by >= y0 && by < y0 + FT::TY) ? (bx - x0) + FT::TX * (by - y0) : -1;
    }
    if (v == 0) sSlot[s * TC + tc] = slot[s];
  }

  // 1. weights of variable v -> nodal values and traces; halo traces
  real w[N];
#pragma unroll
  for (int l = 0; l < N; ++l)
    w[l] = valid ? a.U[(size_t)(v * N + l) * nc + c] : ((v == 0 && l == 0) ? real(1) : real(0));
  {
    real u[Q];
    modal_to_nodal<real, 2, K>(T, w, u);
#pragma unroll
    for (int q = 0; q < Q; ++q) sU[(v * Q + q) * TC + tc] = u[q];
  }
  auto put = [&](real* dst, int s, const real* tr) {
#pragma unroll
    for (int q = 0; q < QF; ++q) dst[((s * NV + v) * QF + q) * TC + tc] = tr[q];
  };
  {
    real tr[QF];
    fused_trace<real, K, 0>(T, w, tr);
    put(sT, 0, tr);
    fused_trace<real, K, 1>(T, w, tr);
    put(sT, 1, tr);
    fused_trace<real, K, 2>(T, w, tr);
    put(sT, 2, tr);
    fused_trace<real, K, 3>(T, w, tr);
    put(sT, 3, tr);
  }
  // the neighbour across side s, outside the tile: its trace on its side s ^ 1
  auto halo = [&](auto sc) {
    constexpr int SD = decltype(sc)::value;
    if (slot[SD] != -1) return;
    const int nb = a.m.nbr[(size_t)SD * nc + c];
    real wn[N], tr[QF];
#pragma unroll
    for (int l = 0; l < N; ++l) wn[l] = a.U[(size_t)(v * N + l) * nc + nb];
    fused_trace<real, K, SD ^ 1>(T, wn, tr);
    put(sH, SD, tr);
  };
  halo(std::integral_constant<int, 0>{});
  halo(std::integral_constant<int, 1>{});
  halo(std::integral_constant<int, 2>{});
  halo(std::integral_constant<int, 3>{});
  __syncthreads();

  // 2. HLLC at the points of every face the tile owns; item (cell, side, point)
  const real gamma = a.gam;
  for (int item = threadIdx.x; item < TC * 4 * QF; item += FT::THREADS) {
    const int ti = item % TC, s = (item / TC) % 4, q = item / (4 * TC);
    const int gxi = x0 + ti % FT::TX, gyi = y0 + ti / FT::TX;
    if (gxi >= nx || gyi >= ny) continue;
    const int sl = sSlot[s * TC + ti];
    if (!(s & 1) && sl >= 0) continue;  // a - side inside the tile: the neighbour's + side
    real uo[NV], un[NV], Fl[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) {
      uo[vv] = sT[((s * NV + vv) * QF + q) * TC + ti];
      un[vv] = sl >= 0 ? sT[(((s ^ 1) * NV + vv) * QF + q) * TC + sl]
                       : (sl == -1 ? sH[((s * NV + vv) * QF + q) * TC + ti] : uo[vv]);
    }
    // the minus state is the + side's trace: this cell's on its + sides
    const real* uL = (s & 1) ? uo : un;
    const real* uR = (s & 1) ? un : uo;
    if (s < 2) hllc_flux<real, 2>(uL, uR, 0, gamma, Fl);
    else hllc_flux<real, 2>(uL, uR, 1, gamma, Fl);
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) sF[((s * NV + vv) * QF + q) * TC + ti] = Fl[vv];
  }

  // 3. point fluxes (the nodal values are read before this thread overwrites them)
  const real g1 = a.gm1;
  for (int q = v; q < Q; q += NV) {
    real u[NV];
#pragma unroll
    for (int vv = 0; vv < NV; ++vv) u[vv] = sU[(vv * Q + q) * TC + tc];
    real f[2][NV];
    euler_flux_all<real, 2>(u, g1, f);
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) sFl[((d * NV + vv) * Q + q) * TC + tc] = f[d][vv];
  }
  __syncthreads();
  if (!valid) return;

  // volume and surface integrals of this variable, then the stage combination
  real acc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l] = real(0);
  {
    real f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = sFl[((0 * NV + v) * Q + q) * TC + tc];
    volume_dir<real, 2, K, 0>(T, f, acc);
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = sFl[((1 * NV + v) * Q + q) * TC + tc];
    volume_dir<real, 2, K, 1>(T, f, acc);
  }
  auto surface = [&](auto sc) {
    constexpr int SD = decltype(sc)::value;
    real fq[QF];
    const int sl = slot[SD];
#pragma unroll
    for (int q = 0; q < QF; ++q)
      fq[q] = (!(SD & 1) && sl >= 0) ? sF[(((SD ^ 1) * NV + v) * QF + q) * TC + sl] : sF[((SD * NV + v) * QF + q) * TC + tc];
    surface_side<real, 2, K, (SD >> 1), (SD & 1)>(T, T.PW, T.PW, fq, real(1), acc);
  };
  surface(std::integral_constant<int, 0>{});
  surface(std::integral_constant<int, 1>{});
  surface(std::integral_constant<int, 2>{});
  surface(std::integral_constant<int, 3>{});
  const int pb = cell_problem(a.m, c);
  const real pre = a.pre_prob ? a.pre_prob[pb] : a.pre[a.m.level[c]];
  stage_epilogue<real, N>(a, c, v, pre * (a.dt ? real(a.dt[pb]) : real(1)), acc, w);
}

template <typename real, int K>
cudaError_t launch_stage_fused(const void* pa, cudaStream_t s) {
  const auto& a = *static_cast<const StageArgs<real>*>(pa);
  using FT = FusedTile<real, K>;
  if (a.m.ncells == 0) return cudaSuccess;
  stage_fused_kernel<real, K><<<FT::blocks(a.m.n[0], a.m.n[1]), FT::THREADS, FT::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <typename real, int K>
cudaError_t prepare_stage_fused() {
  return cudaFuncSetAttribute(stage_fused_kernel<real, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)FusedTile<real, K>::SMEM);
}

}  // namespace dgi
