// Kernel instantiations for 16-bit fingerprints (b in {4, 8, 16}, XOR and
// Offset bucket policies).
#include "cf_launch.cuh"

namespace cfk {

const Ops* ops_f16(int b, int policy) {
  if (policy == 0) {
    switch (b) {
      case 4: return ops_for<Geo<16, 4, 0>>();
      case 8: return ops_for<Geo<16, 8, 0>>();
      case 16: return ops_for<Geo<16, 16, 0>>();
    }
  } else if (policy == 1) {
    switch (b) {
      case 4: return ops_for<Geo<16, 4, 1>>();
      case 8: return ops_for<Geo<16, 8, 1>>();
      case 16: return ops_for<Geo<16, 16, 1>>();
    }
  }
  return nullptr;
}

}  // namespace cfk
