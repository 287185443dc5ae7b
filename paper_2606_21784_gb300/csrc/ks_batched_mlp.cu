// Batched persistent kernel with the policy path, 512 threads per CTA.
#include "ks_batched.cuh"

namespace ks {

#define KS_MLP_BATCH_TU(NT)                                                                                    \
  template <>                                                                                                  \
  __device__ __forceinline__ void dispatch_item_mlp<NT>(const DevParams& P, const BatchArgs& B, uint4 d, uint32_t s0, uint32_t n, \
                                        unsigned char* raw, const MlpCta& mc) {                                \
    switch (d.z & 0xFFFFu) {                                                                                             \
      KS_BATCH_MLP_VARIANTS_##NT(KS_MLP_CASE##NT) default : if (threadIdx.x == 0) atomicOr(P.err, ERR_SHAPE);  \
    }                                                                                                          \
  }                                                                                                            \
  cudaError_t launch_batched_mlp_##NT(const DevParams& p, uint32_t n_steps, const BatchArgs& b, int grid,      \
                                      size_t smem, cudaStream_t st) {                                          \
    batched_mlp_kernel<NT><<<grid, NT, smem, st>>>(p, n_steps, b);                                             \
    return cudaGetLastError();                                                                                 \
  }                                                                                                            \
  const void* batched_mlp_kernel_##NT() { return (const void*)&batched_mlp_kernel<NT>; }

#define KS_MLP_CASE512(ID, GT, AK) \
  case ID:                        \
    run_item_mlp<512, GT, AK>(P, B, d, s0, n, raw, mc); \
    break;

KS_MLP_BATCH_TU(512)

#define KS_ROW(ID, GT, AK) {GT, AK},
extern const int kBatchMlpVariants512[][2] = {KS_BATCH_MLP_VARIANTS_512(KS_ROW)};
#undef KS_ROW
extern const int kBatchMlpVariants512Count = sizeof(kBatchMlpVariants512) / sizeof(kBatchMlpVariants512[0]);

}  // namespace ks
