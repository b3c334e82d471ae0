// Kernel instantiations for dim = 3, k = 0..2, FP64.
#include "dg_kernels.cuh"

namespace dgi {

bool kernel_set_3d_f64(int k, KernelSet* out) {
  switch (k) {
    case 0: *out = make_kernel_set<double, 3, 0>(0); return true;
    case 1: *out = make_kernel_set<double, 3, 1>(0); return true;
    case 2: *out = make_kernel_set<double, 3, 2>(0); return true;
  }
  return false;
}

}  // namespace dgi
