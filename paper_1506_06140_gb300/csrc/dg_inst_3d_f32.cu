// Kernel instantiations for dim = 3, k = 0..2, FP32.
#include "dg_kernels.cuh"

namespace dgi {

bool kernel_set_3d_f32(int k, KernelSet* out) {
  switch (k) {
    case 0: *out = make_kernel_set<float, 3, 0>(1); return true;
    case 1: *out = make_kernel_set<float, 3, 1>(1); return true;
    case 2: *out = make_kernel_set<float, 3, 2>(1); return true;
  }
  return false;
}

}  // namespace dgi
