// Instantiations of the persistent kernel for 128 threads per CTA.
#include "ks_plain.cuh"

namespace ks {
#define KS_VARIANT(NT, AK)                                                                   \
  PlainVariant { NT, AK, &launch_plain<NT, AK>, (const void*)&plain_kernel<NT, AK, false>, \
                 (const void*)&plain_kernel<NT, AK, true> }
extern const PlainVariant kPlainNT128[5] = {KS_VARIANT(128, 1), KS_VARIANT(128, 2), KS_VARIANT(128, 4),
                                        KS_VARIANT(128, 8), KS_VARIANT(128, 16)};
}  // namespace ks
