// Kernel instantiations for dim = 2, k = 0..3, FP32.
#include "dg_kernels.cuh"

namespace dgi {

bool kernel_set_2d_f32(int k, KernelSet* out) {
  switch (k) {
    case 0: *out = make_kernel_set<float, 2, 0>(1); return true;
    case 1: *out = make_kernel_set<float, 2, 1>(1); return true;
    case 2: *out = make_kernel_set<float, 2, 2>(1); return true;
    case 3: *out = make_kernel_set<float, 2, 3>(1); return true;
  }
  return false;
}

}  // namespace dgi
