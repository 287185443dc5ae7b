// Instantiations of the persistent kernel with the policy path (learned
// agents, captures): whole-warpgroup CTAs, plain shared atomics.
#include "ks_plain.cuh"

namespace ks {
// occupancy 1: 128-register cap (two 256-thread or four 128-thread CTAs per SM by registers)
#define KS_MLP_VARIANT(NT, AK, OCC)                                                                      \
  PlainVariant {                                                                                         \
    NT, AK, false, OCC, &launch_plain<NT, AK, false, OCC, true>, (const void*)&plain_kernel<NT, AK, false, OCC, true>, 1 \
  }
extern const PlainVariant kPlainMlp[] = {KS_MLP_VARIANT(128, 16, 0), KS_MLP_VARIANT(128, 16, 1), KS_MLP_VARIANT(256, 8, 0),
                                         KS_MLP_VARIANT(256, 8, 1),  KS_MLP_VARIANT(256, 16, 0), KS_MLP_VARIANT(256, 16, 1),
                                         KS_MLP_VARIANT(512, 4, 0),  KS_MLP_VARIANT(512, 8, 0),  KS_MLP_VARIANT(512, 16, 0),
                                         KS_MLP_VARIANT(1024, 8, 0), KS_MLP_VARIANT(1024, 16, 0)};
extern const int kPlainMlpCount = sizeof(kPlainMlp) / sizeof(kPlainMlp[0]);
}  // namespace ks
