// Instantiations of the persistent kernel for 512 threads per CTA.
#include "ks_plain.cuh"

namespace ks {
#define KS_VARIANT(NT, AK)                                                                   \
  PlainVariant { NT, AK, &launch_plain<NT, AK>, (const void*)&plain_kernel<NT, AK, false>, \
                 (const void*)&plain_kernel<NT, AK, true> }
extern const PlainVariant kPlainNT512[5] = {KS_VARIANT(512, 1), KS_VARIANT(512, 2), KS_VARIANT(512, 4),
                                        KS_VARIANT(512, 8), KS_VARIANT(512, 16)};
}  // namespace ks
