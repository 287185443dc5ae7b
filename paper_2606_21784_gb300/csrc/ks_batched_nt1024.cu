// Batched persistent kernel with 1024 threads per CTA.
#include "ks_batched.cuh"

namespace ks {

template <>
__device__ __forceinline__ void dispatch_item<1024>(const DevParams& P, const BatchArgs& B, uint4 d, uint32_t s0, uint32_t n,
                                   unsigned char* raw) {
  switch (d.z) {
#define KS_CASE(ID, GT, AK) \
  case ID:                  \
    run_item<1024, GT, AK>(P, B, d, s0, n, raw); \
    break;
    KS_BATCH_VARIANTS_1024(KS_CASE)
#undef KS_CASE
    default:
      if (threadIdx.x == 0) atomicOr(P.err, ERR_SHAPE);
  }
}

cudaError_t launch_batched_1024(const DevParams& p, uint32_t n_steps, const BatchArgs& b, int grid, size_t smem,
                               cudaStream_t st) {
  batched_kernel<1024><<<grid, 1024, smem, st>>>(p, n_steps, b);
  return cudaGetLastError();
}

const void* batched_kernel_1024() { return (const void*)&batched_kernel<1024>; }

#define KS_ROW(ID, GT, AK) {GT, AK},
extern const int kBatchVariants1024[][2] = {KS_BATCH_VARIANTS_1024(KS_ROW)};
#undef KS_ROW
extern const int kBatchVariants1024Count = sizeof(kBatchVariants1024) / sizeof(kBatchVariants1024[0]);

}  // namespace ks
