// Instantiations of the persistent kernel with the policy path (learned
// agents, captures): whole-warpgroup CTAs, plain shared atomics.
#include "ks_plain.cuh"

namespace ks {
#define KS_MLP_VARIANT(NT, AK) \
  PlainVariant { NT, AK, false, 0, &launch_plain<NT, AK, false, 0, true>, (const void*)&plain_kernel<NT, AK, false, 0, true>, 1 }
extern const PlainVariant kPlainMlp[] = {KS_MLP_VARIANT(128, 16), KS_MLP_VARIANT(256, 8), KS_MLP_VARIANT(256, 16),
                                         KS_MLP_VARIANT(512, 8),  KS_MLP_VARIANT(512, 16), KS_MLP_VARIANT(1024, 8),
                                         KS_MLP_VARIANT(1024, 16)};
extern const int kPlainMlpCount = sizeof(kPlainMlp) / sizeof(kPlainMlp[0]);
}  // namespace ks
