// Kernel instantiations for the tensor-product basis Q_k: dim = 2, k = 1..3,
// FP64 and FP32 states (stage, timestep, projection and diagnostic kernels).
#include "dg_kernels.cuh"

namespace dgi {

bool kernel_set_2d_tensor(int prec, int k, KernelSet* out) {
  if (prec == 0) {
    switch (k) {
      case 1: *out = make_kernel_set<double, 2, 1, 1>(0); return true;
      case 2: *out = make_kernel_set<double, 2, 2, 1>(0); return true;
      case 3: *out = make_kernel_set<double, 2, 3, 1>(0); return true;
    }
  } else {
    switch (k) {
      case 1: *out = make_kernel_set<float, 2, 1, 1>(1); return true;
      case 2: *out = make_kernel_set<float, 2, 2, 1>(1); return true;
      case 3: *out = make_kernel_set<float, 2, 3, 1>(1); return true;
    }
  }
  return false;
}

}  // namespace dgi
