// Instantiations of the persistent kernel for 1024 threads per CTA.
#include "ks_plain.cuh"

namespace ks {
#define KS_VARIANT(NT, AK, AG, OCC) \
  PlainVariant { NT, AK, AG, OCC, &launch_plain<NT, AK, AG, OCC>, (const void*)&plain_kernel<NT, AK, AG, OCC> }
#define KS_VARIANTS_AK(NT, AK) KS_VARIANT(NT, AK, false, 0), KS_VARIANT(NT, AK, false, 1)
// 4 agents per thread also with the 64-register cap (one 1024-thread CTA per SM, 32 warps)
extern const PlainVariant kPlainNT1024[] = {KS_VARIANTS_AK(1024, 1), KS_VARIANTS_AK(1024, 2), KS_VARIANTS_AK(1024, 4),
                                       KS_VARIANTS_AK(1024, 8), KS_VARIANTS_AK(1024, 16), KS_VARIANT(1024, 4, false, 3)};
extern const int kPlainNT1024Count = sizeof(kPlainNT1024) / sizeof(kPlainNT1024[0]);
}  // namespace ks
