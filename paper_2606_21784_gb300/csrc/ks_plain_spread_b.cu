// Instantiations of the persistent kernel whose markets spread their agents
// over the CTA (512- and 1024-thread CTAs, 128-register cap class).
#include "ks_plain.cuh"

namespace ks {
#define KS_SPREAD_VARIANT(NT, AK)                                                                       \
  PlainVariant {                                                                                        \
    NT, AK, false, 1, &launch_plain<NT, AK, false, 1, false, true>,                                     \
        (const void*)&plain_kernel<NT, AK, false, 1, false, true>, 0, 1                                 \
  }
extern const PlainVariant kPlainSpreadB[] = {KS_SPREAD_VARIANT(512, 8), KS_SPREAD_VARIANT(512, 16),
                                             KS_SPREAD_VARIANT(1024, 8), KS_SPREAD_VARIANT(1024, 16)};
extern const int kPlainSpreadBCount = sizeof(kPlainSpreadB) / sizeof(kPlainSpreadB[0]);
}  // namespace ks
