// Instantiations of the persistent kernel for 128 threads per CTA.
#include "ks_plain.cuh"

namespace ks {
#define KS_VARIANT(NT, AK, AG, OCC) \
  PlainVariant { NT, AK, AG, OCC, &launch_plain<NT, AK, AG, OCC>, (const void*)&plain_kernel<NT, AK, AG, OCC> }
#define KS_VARIANTS_AK(NT, AK) KS_VARIANT(NT, AK, false, 0), KS_VARIANT(NT, AK, false, 1)
// small agent tiles also with the 85-register cap (three 256-thread or six 128-thread CTAs per SM)
#define KS_VARIANTS_AK3(NT, AK) KS_VARIANTS_AK(NT, AK), KS_VARIANT(NT, AK, false, 2)
extern const PlainVariant kPlainNT128[] = {KS_VARIANTS_AK3(128, 1), KS_VARIANTS_AK3(128, 2), KS_VARIANTS_AK3(128, 4),
                                       KS_VARIANTS_AK(128, 8), KS_VARIANTS_AK(128, 16)};
extern const int kPlainNT128Count = sizeof(kPlainNT128) / sizeof(kPlainNT128[0]);
}  // namespace ks
