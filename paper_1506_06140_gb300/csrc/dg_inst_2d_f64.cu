// Kernel instantiations for dim = 2, k = 0..3, FP64.
#include "dg_kernels.cuh"

namespace dgi {

bool kernel_set_2d_f64(int k, KernelSet* out) {
  switch (k) {
    case 0: *out = make_kernel_set<double, 2, 0>(0); return true;
    case 1: *out = make_kernel_set<double, 2, 1>(0); return true;
    case 2: *out = make_kernel_set<double, 2, 2>(0); return true;
    case 3: *out = make_kernel_set<double, 2, 3>(0); return true;
  }
  return false;
}

}  // namespace dgi
