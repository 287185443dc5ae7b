// Instantiations of the persistent kernel for 64 threads per CTA.
#include "ks_plain.cuh"

namespace ks {
#define KS_VARIANT(NT, AK)                                                                   \
  PlainVariant { NT, AK, &launch_plain<NT, AK>, (const void*)&plain_kernel<NT, AK, false>, \
                 (const void*)&plain_kernel<NT, AK, true> }
extern const PlainVariant kPlainNT64[5] = {KS_VARIANT(64, 1), KS_VARIANT(64, 2), KS_VARIANT(64, 4),
                                        KS_VARIANT(64, 8), KS_VARIANT(64, 16)};
}  // namespace ks
