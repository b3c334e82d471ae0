// dg_totals_noalloc: the conserved-totals reduction without any device
// allocation and without a handle.
//
// Who needs it: code that cannot call cudaMalloc -- for instance a host
// application that owns every device allocation and forbids libraries from
// allocating, or code running while a stream is captured in global mode,
// where allocation calls are not permitted.  Such callers cannot create a
// dg_handle (dg_create allocates its tables and scratch), yet may hold a
// state array and need its totals.  The per-block partial sums, which the
// handle-based dg_totals keeps in handle-owned scratch, live here in one
// file-scope device array of fixed size instead.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "dg.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxVars = 5;
constexpr int64_t kMaxCells = DG_NOALLOC_MAX_CELLS;
constexpr int kMaxBlocks = (int)((kMaxCells + kThreads - 1) / kThreads);

// Scratch: one partial sum per (block, variable).  Every GPU that loads the
// library holds this array until the process exits.  Each block writes its
// own slots before the second pass reads them, so nothing needs clearing.
static __device__ __align__(256) double g_partials[kMaxBlocks * kMaxVars];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {};

// Same fixed order as the handle-based reduction: a shuffle-down tree within
// each warp, then one over the warps' sums; valid in thread 0.
__device__ __forceinline__ double block_sum(double x, double* sh) {
  constexpr unsigned full = 0xffffffffu;
  constexpr int NW = kThreads / 32;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(full, x, o);
  if (l == 0) sh[w] = x;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = l < NW ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(full, r, o);
  }
  __syncthreads();
  return r;
}

template <typename real>
__global__ void __launch_bounds__(kThreads)
    totals_partials(const real* W, int nv, int nb, int nc, int dim, double dx0,
                    const int32_t* levels, double* partial) {
  __shared__ double sh[kThreads];
  const int c = blockIdx.x * kThreads + threadIdx.x;
  double vol = 0.0;
  if (c < nc) {
    const double dx = ldexp(dx0, levels ? -(int)levels[c] : 0);
    vol = dim == 2 ? dx * dx : dx * dx * dx;
  }
  for (int v = 0; v < nv; ++v) {
    const double x = (c < nc) ? vol * (double)W[(size_t)v * nb * nc + c] : 0.0;
    const double s = block_sum(x, sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * nv + v] = s;
  }
}

// one warp per variable, the order of the handle-based final pass
__global__ void totals_final(const double* partial, int nblocks, int nv, double* out) {
  const int v = blockIdx.x, l = threadIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int b = l; b < nblocks; b += 32) s += partial[(size_t)b * nv + v];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (l == 0) out[v] = s;
}

// Device address of the scratch array on the current device (set-up once
// per device; the host-side symbol itself is not a device address).
cudaError_t scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

// Launches through cudaLaunchKernel, whose return value is the status of
// this launch alone: cudaGetLastError would also return (and clear) an
// earlier, unrelated error of the calling thread.
template <typename real>
cudaError_t launch_partials(int nblocks, cudaStream_t s, const void* W, int nv, int nb, int nc,
                            int dim, double dx0, const int32_t* levels, double* partial) {
  const real* Wr = static_cast<const real*>(W);
  void* args[] = {(void*)&Wr, (void*)&nv, (void*)&nb, (void*)&nc, (void*)&dim, (void*)&dx0,
                  (void*)&levels, (void*)&partial};
  return cudaLaunchKernel((const void*)totals_partials<real>, dim3(nblocks), dim3(kThreads), args, 0, s);
}

}  // namespace

extern "C" int dg_totals_noalloc(int dim, int n_basis, int64_t n_cells, int precision, double dx0,
                                 const int32_t* levels_dev, const void* W_dev, double* totals_dev,
                                 void* stream) {
  if (dim != 2 && dim != 3) return DG_ERR_ARG;
  if (n_basis < 1 || n_cells < 0 || !(dx0 > 0.0) || !W_dev || !totals_dev) return DG_ERR_ARG;
  // the state's element type: double for DG_FP64 and the FP64-state mixed
  // modes, float for DG_FP32 and DG_FP32_TC
  const bool dbl = precision == DG_FP64 || precision == DG_MIXED || precision == DG_MIXED_TC;
  if (!dbl && precision != DG_FP32 && precision != DG_FP32_TC) return DG_ERR_ARG;
  if (n_cells > kMaxCells) return DG_ERR_ARG;  // beyond the fixed scratch
  int nv = dim + 2;
  const int nc = (int)n_cells;
  int nblocks = (nc + kThreads - 1) / kThreads;
  double* partial = nullptr;
  if (scratch_on_current_device(&partial) != cudaSuccess) return DG_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nblocks > 0) {
    const cudaError_t e =
        dbl ? launch_partials<double>(nblocks, s, W_dev, nv, n_basis, nc, dim, dx0, levels_dev, partial)
            : launch_partials<float>(nblocks, s, W_dev, nv, n_basis, nc, dim, dx0, levels_dev, partial);
    if (e != cudaSuccess) return DG_ERR_CUDA;
  }
  void* args[] = {(void*)&partial, (void*)&nblocks, (void*)&nv, (void*)&totals_dev};
  return cudaLaunchKernel((const void*)totals_final, dim3(nv), dim3(32), args, 0, s) == cudaSuccess
             ? DG_OK
             : DG_ERR_CUDA;
}
