// ks_probe.cu -- roofline probe kernels (see kineticsim_probe.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include "kineticsim_probe.h"
#include "ks_device.cuh"
#include "ks_mlp.cuh"

namespace ks {

constexpr int PROBE_THREADS = 256;

// Eight red.shared.add.u32 per iteration; lane l of every warp always hits
// bank l, so no two lanes of a warp conflict.
__global__ void __launch_bounds__(PROBE_THREADS) probe_smem_red(uint32_t iters, uint64_t* sink) {
  __shared__ uint32_t buf[8][PROBE_THREADS];
#pragma unroll
  for (int j = 0; j < 8; ++j) buf[j][threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) atomicAdd(&buf[j][threadIdx.x], it + (uint32_t)j);
  }
  __syncthreads();
  uint64_t acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc += buf[j][threadIdx.x];
  sink[(size_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = acc;
}

// Eight independent chains acc = lo32(acc) * C + acc (one mad.wide.u32 each).
__global__ void __launch_bounds__(PROBE_THREADS) probe_mul_wide(uint32_t iters, uint64_t* sink) {
  uint64_t acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = (uint64_t)(threadIdx.x + 977u * j + blockIdx.x);
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = (uint64_t)(uint32_t)acc[j] * (uint64_t)PH_MA + acc[j];
  }
  uint64_t x = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) x ^= acc[j];
  sink[(size_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = x;
}

// Eight independent chains x = hi(x * C) ^ lo(x * C) ^ j: one 32 x 32 -> 64 product
// each, as a high-word and a low-word multiply (the form the Philox rounds use).
__global__ void __launch_bounds__(PROBE_THREADS) probe_mul_hilo(uint32_t iters, uint64_t* sink) {
  uint32_t x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x + 977u * j + blockIdx.x;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = __umulhi(x[j], PH_MA) ^ (x[j] * PH_MA) ^ (uint32_t)j;
  }
  uint64_t acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc = acc * 31u + x[j];
  sink[(size_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = acc;
}

// The persistent kernel's per-agent draw (StepKey + step_draw_x0), one block per iteration.
__global__ void __launch_bounds__(PROBE_THREADS) probe_philox(uint32_t iters, uint64_t* sink) {
  uint32_t rk[20];
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = 0x1234567u + (uint32_t)r * PH_WA;
    rk[2 * r + 1] = 0x89abcdefu + (uint32_t)r * PH_WB;
  }
  const StepKey sk = step_key(7u, blockIdx.x, 0u, rk);
  uint32_t x = 0;
  const uint32_t base = threadIdx.x;
  for (uint32_t it = 0; it < iters; ++it) {
    const uint4 w = step_draw_x0(sk, sk.c0 ^ (base + it * PROBE_THREADS), rk);
    x ^= w.x ^ w.y ^ w.z ^ w.w;
  }
  sink[(size_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = x;
}

// One warpgroup runs the policy path's bounded layer wait on an mbarrier that
// nothing ever arrives at (no tensor-core operation is issued, none is in
// flight): the wait must give up after its poll limit, record ERR_MLP_WAIT in
// the error word and return; a second wait of the aborted warpgroup must not
// poll again.  sink[0] (as uint32) receives the error word.
__global__ void __launch_bounds__(128) probe_wait_timeout(uint32_t* sink) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t err;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1u);
    err = 0u;
  }
  __syncthreads();
  MlpWG g;
  g.bar = &bar;
  g.tmem = 0u;
  g.bar_id = 1;
  g.phase = 0u;
  g.abort = false;
  g.wg = 0;
  g.nwg = 1;
  mlp_wait_bounded(g, &err);
  const bool first = g.abort;
  mlp_wait_bounded(g, &err);
  __syncthreads();
  if (threadIdx.x == 0) {
    sink[0] = err;
    sink[1] = first && g.abort ? 1u : 0u;
  }
}

}  // namespace ks

namespace ks {
double launch_probe_sm64(uint32_t blocks, uint32_t iters, uint64_t* sink, cudaStream_t st);
}

extern "C" ks_status ks_probe(int kind, uint32_t blocks, uint32_t iters, void* sink, void* stream, double* ops) {
  if (!sink || !ops || blocks == 0) return KS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const double lanes = (double)blocks * ks::PROBE_THREADS * (double)iters;
  switch (kind) {
    case KS_PROBE_SMEM_RED:
      ks::probe_smem_red<<<blocks, ks::PROBE_THREADS, 0, st>>>(iters, (uint64_t*)sink);
      *ops = lanes * 8.0;
      break;
    case KS_PROBE_MUL_WIDE:
      ks::probe_mul_wide<<<blocks, ks::PROBE_THREADS, 0, st>>>(iters, (uint64_t*)sink);
      *ops = lanes * 8.0;
      break;
    case KS_PROBE_PHILOX:
      ks::probe_philox<<<blocks, ks::PROBE_THREADS, 0, st>>>(iters, (uint64_t*)sink);
      *ops = lanes;
      break;
    case KS_PROBE_MUL_HILO:
      ks::probe_mul_hilo<<<blocks, ks::PROBE_THREADS, 0, st>>>(iters, (uint64_t*)sink);
      *ops = lanes * 8.0;
      break;
    case KS_PROBE_SPLITMIX:
      *ops = ks::launch_probe_sm64(blocks, iters, (uint64_t*)sink, st);
      break;
    case KS_PROBE_WAIT_TIMEOUT:
      ks::probe_wait_timeout<<<1, 128, 0, st>>>((uint32_t*)sink);
      *ops = 1.0;
      break;
    default:
      return KS_ERR_INVALID_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? KS_OK : KS_ERR_CUDA;
}
