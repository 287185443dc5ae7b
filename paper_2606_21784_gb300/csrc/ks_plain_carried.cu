// Instantiations of the persistent kernel compiled for carried books only
// (128-register cap, one full shape per market): with the book mode a
// compile-time constant, the cancellation threshold and the mask of what an
// order word keeps fold into the code, and the marginal rationing sits behind
// a warp vote.  The launch takes these for an ensemble that carries its book
// when the shape is full (no spreading); the state is the same bit for bit.
#include "ks_plain.cuh"

namespace ks {
#define KS_CARRIED_VARIANT(NT, AK)                                                                      \
  PlainVariant {                                                                                        \
    NT, AK, false, 1, &launch_plain<NT, AK, false, 1, false, false, 1>,                                 \
        (const void*)&plain_kernel<NT, AK, false, 1, false, false, 1>, 0, 0, 1                          \
  }
extern const PlainVariant kPlainCarried[] = {KS_CARRIED_VARIANT(128, 8), KS_CARRIED_VARIANT(128, 16),
                                             KS_CARRIED_VARIANT(256, 8), KS_CARRIED_VARIANT(256, 16),
                                             KS_CARRIED_VARIANT(512, 8), KS_CARRIED_VARIANT(512, 16)};
extern const int kPlainCarriedCount = sizeof(kPlainCarried) / sizeof(kPlainCarried[0]);
}  // namespace ks
