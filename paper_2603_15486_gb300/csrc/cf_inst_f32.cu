// Kernel instantiations for 32-bit fingerprints (b in {4, 8, 16}, XOR and
// Offset bucket policies).
#include "cf_launch.cuh"

namespace cfk {

const Ops* ops_f32(int b, int policy) {
  if (policy == 0) {
    switch (b) {
      case 4: return ops_for<Geo<32, 4, 0>>();
      case 8: return ops_for<Geo<32, 8, 0>>();
      case 16: return ops_for<Geo<32, 16, 0>>();
    }
  } else if (policy == 1) {
    switch (b) {
      case 4: return ops_for<Geo<32, 4, 1>>();
      case 8: return ops_for<Geo<32, 8, 1>>();
      case 16: return ops_for<Geo<32, 16, 1>>();
    }
  }
  return nullptr;
}

}  // namespace cfk
