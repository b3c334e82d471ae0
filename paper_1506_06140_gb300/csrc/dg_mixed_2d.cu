// Mixed-precision stage kernels (FP64 state, FP32 right-hand side in
// perturbation form) for dim = 2, k = 0..3, with the tensor-core cell kernel
// for k = 1..3.
#include "dg_tc.cuh"

namespace dgi {

template <int K>
MixedSet make_mixed_set_2d() {
  MixedSet ms = make_mixed_set<2, K>();
  if constexpr (K >= 1) {
    ms.cell_tc = &launch_cell_tc<K, true>;
    ms.prepare_tc = &prepare_cell_tc<K, true>;
    ms.fill_tc = &fill_tc_tables<K>;
  }
  return ms;
}

bool mixed_set_2d(int k, MixedSet* out) {
  switch (k) {
    case 0: *out = make_mixed_set_2d<0>(); return true;
    case 1: *out = make_mixed_set_2d<1>(); return true;
    case 2: *out = make_mixed_set_2d<2>(); return true;
    case 3: *out = make_mixed_set_2d<3>(); return true;
  }
  return false;
}

}  // namespace dgi
