// Instantiations of the persistent kernel for 256 threads per CTA.
#include "ks_plain.cuh"

namespace ks {
#define KS_VARIANT(NT, AK)                                                                   \
  PlainVariant { NT, AK, &launch_plain<NT, AK>, (const void*)&plain_kernel<NT, AK, false>, \
                 (const void*)&plain_kernel<NT, AK, true> }
extern const PlainVariant kPlainNT256[5] = {KS_VARIANT(256, 1), KS_VARIANT(256, 2), KS_VARIANT(256, 4),
                                        KS_VARIANT(256, 8), KS_VARIANT(256, 16)};
}  // namespace ks
