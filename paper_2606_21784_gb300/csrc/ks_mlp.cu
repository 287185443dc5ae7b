// ks_mlp.cu -- standalone forward of the agent policy for feature rows given
// by the caller: the step loop's tensor-core tile code for layers 2-3, the
// full FP32 first layer on the CUDA cores.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kineticsim.h"
#include "ks_mlp.cuh"

namespace ks {

constexpr int FWD_NWG = 2;  // warpgroups per CTA (MLP_TMEM_COLS TMEM columns each)

__host__ __device__ constexpr uint32_t fwd_smem_bytes() {
  return ((MLP_SM_BYTES + 127u) & ~127u) + 8 * FWD_NWG + 16;
}
// Dynamic shared memory requested per CTA: enough that at most two CTAs share
// an SM, so their TMEM (2 x 256 columns) never exceeds the SM's 512.
constexpr uint32_t FWD_SMEM_REQUEST = 100u * 1024u;

__global__ void __launch_bounds__(128 * FWD_NWG, 1)
    mlp_forward_kernel(const unsigned char* blob, const float* X, int64_t n, float* Z, uint32_t* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sw = sm;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + ((MLP_SM_BYTES + 127u) & ~127u));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + FWD_NWG);
  const int wg = (int)threadIdx.x / 128;
  const int r = (int)threadIdx.x & 127;
  if (threadIdx.x < 32) {
    tmem_alloc(tslot, MLP_TMEM_COLS * FWD_NWG);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < FWD_NWG; ++i) mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  mlp_load_weights(blob, sw, (int)threadIdx.x, (int)blockDim.x);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  MlpWG g;
  g.bar = &bars[wg];
  g.tmem = *tslot + (uint32_t)(wg * MLP_TMEM_COLS);
  g.bar_id = 1 + wg;
  g.phase = 0;
  g.abort = false;
  g.wg = wg;
  g.nwg = FWD_NWG;
  const int64_t ntiles = (n + 127) / 128;
  for (int64_t tile = (int64_t)blockIdx.x * FWD_NWG + wg; tile < ntiles; tile += (int64_t)gridDim.x * FWD_NWG) {
    const int64_t row = tile * 128 + r;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) x[i] = row < n ? X[row * MLP_IN + i] : 0.0f;
    float h1[MLP_H];
    mlp_layer1(sw, x, h1);
    float z[MLP_OUT];
    mlp_tile_forward(g, sw, h1, z, err);
    if (row < n) {
#pragma unroll
      for (int i = 0; i < MLP_OUT; ++i) Z[row * MLP_OUT + i] = z[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(*tslot, MLP_TMEM_COLS * FWD_NWG);
  }
}

}  // namespace ks

extern "C" ks_status ks_mlp_forward(const void* params, const float* X, int64_t n, float* Z, uint32_t* err,
                                    void* stream) {
  if (!params || !err || n < 0 || (n > 0 && (!X || !Z))) return KS_ERR_INVALID_ARG;
  if (((uintptr_t)params & 15u) != 0) return KS_ERR_INVALID_ARG;
  if (n == 0) return KS_OK;
  static_assert(ks::fwd_smem_bytes() <= ks::FWD_SMEM_REQUEST, "smem");
  const size_t smem = ks::FWD_SMEM_REQUEST;
  cudaError_t e = cudaFuncSetAttribute(ks::mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return KS_ERR_CUDA;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (n + 127) / 128;
  // TMEM: 256 columns per CTA; the shared-memory request keeps at most 2 CTAs on an SM (512 columns)
  const int64_t want = (ntiles + ks::FWD_NWG - 1) / ks::FWD_NWG;
  const int grid = (int)(want < (int64_t)sms * 2 ? want : (int64_t)sms * 2);
  ks::mlp_forward_kernel<<<grid, 128 * ks::FWD_NWG, smem, (cudaStream_t)stream>>>(
      (const unsigned char*)params, X, n, Z, err);
  return cudaGetLastError() == cudaSuccess ? KS_OK : KS_ERR_CUDA;
}
