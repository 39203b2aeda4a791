// Multi-filter launch variants for 8-bit fingerprints.
#include "cf_batch.cuh"

namespace cfk {

const BatchVariant* batch_variants_f8(int b, int policy, int* count) {
  *count = 0;
  if (policy == 0) {
    switch (b) {
      case 4: return BatchVariants<Geo<8, 4, 0>>::get(count);
      case 8: return BatchVariants<Geo<8, 8, 0>>::get(count);
      case 16: return BatchVariants<Geo<8, 16, 0>>::get(count);
    }
  } else if (policy == 1) {
    switch (b) {
      case 4: return BatchVariants<Geo<8, 4, 1>>::get(count);
      case 8: return BatchVariants<Geo<8, 8, 1>>::get(count);
      case 16: return BatchVariants<Geo<8, 16, 1>>::get(count);
    }
  }
  return nullptr;
}

}  // namespace cfk
