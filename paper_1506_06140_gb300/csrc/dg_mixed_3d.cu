// Mixed-precision stage kernels (FP64 state, FP32 right-hand side in
// perturbation form) for dim = 3, k = 0..3.
#include "dg_mixed.cuh"

namespace dgi {

bool mixed_set_3d(int k, MixedSet* out) {
  switch (k) {
    case 0: *out = make_mixed_set<3, 0>(); return true;
    case 1: *out = make_mixed_set<3, 1>(); return true;
    case 2: *out = make_mixed_set<3, 2>(); return true;
    case 3: *out = make_mixed_set<3, 3>(); return true;
  }
  return false;
}

}  // namespace dgi
