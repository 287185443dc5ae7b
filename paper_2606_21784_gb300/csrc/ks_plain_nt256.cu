// Instantiations of the persistent kernel for 256 threads per CTA.
#include "ks_plain.cuh"

namespace ks {
#define KS_VARIANT(NT, AK, AG, OCC) \
  PlainVariant { NT, AK, AG, OCC, &launch_plain<NT, AK, AG, OCC>, (const void*)&plain_kernel<NT, AK, AG, OCC> }
#define KS_VARIANTS_AK(NT, AK) KS_VARIANT(NT, AK, false, 0), KS_VARIANT(NT, AK, false, 1)
// small agent tiles also with the 85-register cap (three 256-thread CTAs per SM)
#define KS_VARIANTS_AK3(NT, AK) KS_VARIANTS_AK(NT, AK), KS_VARIANT(NT, AK, false, 2)
extern const PlainVariant kPlainNT256[] = {KS_VARIANTS_AK3(256, 1), KS_VARIANTS_AK3(256, 2), KS_VARIANTS_AK3(256, 4),
                                       KS_VARIANTS_AK(256, 8), KS_VARIANTS_AK(256, 16), KS_VARIANT(256, 16, true, 0), KS_VARIANT(256, 8, true, 0)};
extern const int kPlainNT256Count = sizeof(kPlainNT256) / sizeof(kPlainNT256[0]);
}  // namespace ks
