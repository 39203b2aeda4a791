// Multi-filter launch variants for 32-bit fingerprints.
#include "cf_batch.cuh"

namespace cfk {

const BatchVariant* batch_variants_f32(int b, int policy, int* count) {
  *count = 0;
  if (policy == 0) {
    switch (b) {
      case 4: return BatchVariants<Geo<32, 4, 0>>::get(count);
      case 8: return BatchVariants<Geo<32, 8, 0>>::get(count);
      case 16: return BatchVariants<Geo<32, 16, 0>>::get(count);
    }
  } else if (policy == 1) {
    switch (b) {
      case 4: return BatchVariants<Geo<32, 4, 1>>::get(count);
      case 8: return BatchVariants<Geo<32, 8, 1>>::get(count);
      case 16: return BatchVariants<Geo<32, 16, 1>>::get(count);
    }
  }
  return nullptr;
}

}  // namespace cfk
