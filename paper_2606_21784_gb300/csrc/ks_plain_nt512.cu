// Instantiations of the persistent kernel for 512 threads per CTA.
#include "ks_plain.cuh"

namespace ks {
#define KS_VARIANT(NT, AK, AG, OCC) \
  PlainVariant { NT, AK, AG, OCC, &launch_plain<NT, AK, AG, OCC>, (const void*)&plain_kernel<NT, AK, AG, OCC> }
#define KS_VARIANTS_AK(NT, AK) KS_VARIANT(NT, AK, false, 0), KS_VARIANT(NT, AK, false, 1)
// 8 agents per thread also with the 64-register cap (two 512-thread CTAs per SM)
extern const PlainVariant kPlainNT512[] = {KS_VARIANTS_AK(512, 1), KS_VARIANTS_AK(512, 2), KS_VARIANTS_AK(512, 4),
                                       KS_VARIANTS_AK(512, 8), KS_VARIANTS_AK(512, 16), KS_VARIANT(512, 8, true, 0), KS_VARIANT(512, 16, true, 0),
                                       KS_VARIANT(512, 8, false, 3)};
extern const int kPlainNT512Count = sizeof(kPlainNT512) / sizeof(kPlainNT512[0]);
}  // namespace ks
