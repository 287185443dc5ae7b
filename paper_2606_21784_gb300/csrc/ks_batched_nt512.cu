// Batched persistent kernel with 512 threads per CTA.
#include "ks_batched.cuh"

namespace ks {

template <>
__device__ __forceinline__ void dispatch_item<512>(const DevParams& P, const BatchArgs& B, uint4 d, uint32_t s0, uint32_t n,
                                   unsigned char* raw) {
  switch (d.z) {
#define KS_CASE(ID, GT, AK) \
  case ID:                  \
    run_item<512, GT, AK>(P, B, d, s0, n, raw); \
    break;
    KS_BATCH_VARIANTS_512(KS_CASE)
#undef KS_CASE
    default:
      if (threadIdx.x == 0) atomicOr(P.err, ERR_SHAPE);
  }
}

cudaError_t launch_batched_512(const DevParams& p, uint32_t n_steps, const BatchArgs& b, int grid, size_t smem,
                               cudaStream_t st) {
  batched_kernel<512><<<grid, 512, smem, st>>>(p, n_steps, b);
  return cudaGetLastError();
}

const void* batched_kernel_512() { return (const void*)&batched_kernel<512>; }

#define KS_ROW(ID, GT, AK) {GT, AK},
extern const int kBatchVariants512[][2] = {KS_BATCH_VARIANTS_512(KS_ROW)};
#undef KS_ROW
extern const int kBatchVariants512Count = sizeof(kBatchVariants512) / sizeof(kBatchVariants512[0]);

}  // namespace ks
