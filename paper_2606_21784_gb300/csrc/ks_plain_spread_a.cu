// Instantiations of the persistent kernel whose markets spread their agents
// over the CTA (128- and 256-thread CTAs, 128-register cap): the launch takes
// these when a shape holds more agents than the ensemble's largest market
// (measured: 128 x 4, which spreads at most a quarter, gained nothing).
#include "ks_plain.cuh"

namespace ks {
#define KS_SPREAD_VARIANT(NT, AK)                                                                       \
  PlainVariant {                                                                                        \
    NT, AK, false, 1, &launch_plain<NT, AK, false, 1, false, true>,                                     \
        (const void*)&plain_kernel<NT, AK, false, 1, false, true>, 0, 1                                 \
  }
extern const PlainVariant kPlainSpreadA[] = {KS_SPREAD_VARIANT(128, 8), KS_SPREAD_VARIANT(128, 16),
                                             KS_SPREAD_VARIANT(256, 8), KS_SPREAD_VARIANT(256, 16)};
extern const int kPlainSpreadACount = sizeof(kPlainSpreadA) / sizeof(kPlainSpreadA[0]);
}  // namespace ks
