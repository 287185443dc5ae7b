// Instantiations of the persistent kernel for 1024 threads per CTA.
#include "ks_plain.cuh"

namespace ks {
#define KS_VARIANT(NT, AK)                                                                   \
  PlainVariant { NT, AK, &launch_plain<NT, AK>, (const void*)&plain_kernel<NT, AK, false>, \
                 (const void*)&plain_kernel<NT, AK, true> }
extern const PlainVariant kPlainNT1024[5] = {KS_VARIANT(1024, 1), KS_VARIANT(1024, 2), KS_VARIANT(1024, 4),
                                        KS_VARIANT(1024, 8), KS_VARIANT(1024, 16)};
}  // namespace ks
