// Small helper kernels shared by all schemes, and the kernel-set dispatch.
#include <algorithm>
#include <mutex>

#include "dg_internal.h"
#include "dg_physics.cuh"

namespace dgi {

bool kernel_set_2d_f64(int k, KernelSet* out);
bool kernel_set_2d_f32(int k, KernelSet* out);
bool kernel_set_3d_f64(int k, KernelSet* out);
bool kernel_set_3d_f32(int k, KernelSet* out);

bool kernel_set_2d_tensor(int prec, int k, KernelSet* out);

// basis 1 (tensor product Q_k): 2D, k = 1..3; at k = 0 both bases are the constant
const KernelSet* kernel_set(int prec, int dim, int k, int basis) {
  static KernelSet sets[2][2][4];
  static bool have[2][2][4] = {};
  static KernelSet tsets[2][4];
  static bool thave[2][4] = {};
  static std::mutex mu;
  if (prec < 0 || prec > 1 || (dim != 2 && dim != 3) || k < 0 || k > 3) return nullptr;
  if (basis != 0 && (basis != 1 || dim != 2)) return nullptr;
  if (k == 0) basis = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (basis == 1) {
    KernelSet& ts = tsets[prec][k];
    if (!thave[prec][k]) {
      if (!kernel_set_2d_tensor(prec, k, &ts)) return nullptr;
      thave[prec][k] = true;
    }
    return &ts;
  }
  KernelSet& ks = sets[prec][dim - 2][k];
  if (!have[prec][dim - 2][k]) {
    const bool ok = dim == 2 ? (prec == 0 ? kernel_set_2d_f64(k, &ks) : kernel_set_2d_f32(k, &ks))
                             : (prec == 0 ? kernel_set_3d_f64(k, &ks) : kernel_set_3d_f32(k, &ks));
    if (!ok) return nullptr;
    have[prec][dim - 2][k] = true;
  }
  return &ks;
}

bool mixed_set_2d(int k, MixedSet* out);
bool mixed_set_3d(int k, MixedSet* out);

const MixedSet* mixed_set(int dim, int k) {
  static MixedSet sets[2][4];
  static bool have[2][4] = {};
  static std::mutex mu;
  if ((dim != 2 && dim != 3) || k < 0 || k > 3) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  MixedSet& ms = sets[dim - 2][k];
  if (!have[dim - 2][k]) {
    const bool ok = dim == 2 ? mixed_set_2d(k, &ms) : mixed_set_3d(k, &ms);
    if (!ok) return nullptr;
    have[dim - 2][k] = true;
  }
  return &ms;
}

template <typename T>
__global__ void fill_kernel(T* dst, size_t n, T value) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = value;
}

cudaError_t launch_fill(void* dst, size_t n, double value, int esize, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (esize == 8) fill_kernel<double><<<grid, 256, 0, s>>>(static_cast<double*>(dst), n, value);
  else fill_kernel<float><<<grid, 256, 0, s>>>(static_cast<float*>(dst), n, (float)value);
  return cudaGetLastError();
}

__global__ void set_scalar_kernel(double* dst, int n, double value) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = value;
}

cudaError_t launch_set_scalar(double* dst, int n, double value, cudaStream_t s) {
  set_scalar_kernel<<<(n + 255) / 256, 256, 0, s>>>(dst, n, value);
  return cudaGetLastError();
}

// the largest signal speed of each problem was accumulated as the bit
// pattern of a non-negative double; dt = factor / speed
__global__ void dt_finalize_kernel(const unsigned long long* bits, int nprob, double factor,
                                   double* dt, double* dt_copy) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nprob; p += gridDim.x * blockDim.x) {
    const double speed = __longlong_as_double((long long)bits[p]);
    const double v = speed > 0.0 ? factor / speed : 0.0;
    dt[p] = v;
    if (dt_copy) dt_copy[p] = v;
  }
}

__global__ void convert_kernel(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

cudaError_t launch_convert(const double* src, void* dst, size_t n, int esize, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (esize == 8) return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  const size_t blocks = std::min<size_t>((n + 255) / 256, 152 * 16);
  convert_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, static_cast<float*>(dst), n);
  return cudaGetLastError();
}

cudaError_t launch_dt_finalize(const unsigned long long* bits, int nprob, double factor,
                               double* dt, double* dt_copy, cudaStream_t s) {
  dt_finalize_kernel<<<(nprob + 255) / 256, 256, 0, s>>>(bits, nprob, factor, dt, dt_copy);
  return cudaGetLastError();
}

__global__ void flux_math_kernel(int op, const double* x, double* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = op == 0 ? recip(x[i])
             : op == 1 ? sqrt_pos(x[i])
             : op == 2 ? (double)recip((float)x[i])
                       : (double)sqrt_pos((float)x[i]);
}

cudaError_t launch_flux_math(int op, const double* x, double* out, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t b = (n + 255) / 256;
  flux_math_kernel<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, s>>>(op, x, out, n);
  return cudaGetLastError();
}

}  // namespace dgi
