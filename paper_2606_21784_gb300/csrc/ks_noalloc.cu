// ks_noalloc.cu -- ks_step_n_noalloc: the batched persistent launch with its
// scratch in library-owned static device memory.
//
// The batched kernel needs scratch besides the simulation state: the work
// schedule (markets grouped into work items, longest first) and the ticket
// counter from which CTAs take items.  ks_step_n keeps both in the workspace
// the caller allocated.  Callers that cannot allocate device memory for it
// (an allocator that is capped or frozen, code that only hands out its own
// input and output buffers) use this entry point instead: the schedule and the
// ticket live in the static array below, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "kineticsim.h"
#include "ks_batched.cuh"
#include "ks_internal.h"

namespace ks {

ks_status internal_batched_schedule(const ks_ensemble* e, const uint32_t** order, const uint4** items,
                                    uint32_t* n_markets, uint32_t* n_items);
ks_status internal_launch_batched(ks_ensemble* e, uint32_t n_steps, const BatchArgs& b, cudaStream_t st);
int internal_device(const ks_ensemble* e);

// Layout (32-bit words): [0, 64) ticket and padding, then the market order
// (KS_NOALLOC_MAX_MARKETS words), then the work items (4 words each).
constexpr size_t NA_ORDER = 64;
constexpr size_t NA_ITEMS = NA_ORDER + KS_NOALLOC_MAX_MARKETS;
constexpr size_t NA_WORDS = NA_ITEMS + 4 * (size_t)KS_NOALLOC_MAX_MARKETS;
static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

constexpr int NA_MAX_DEVICES = 64;
static uint32_t* g_scratch_addr[NA_MAX_DEVICES];
static std::mutex g_scratch_mu;

// Device address of the static array on device `dev` (which is current),
// looked up on the first call on that device and kept for the process.  A
// cudaDeviceReset unloads the module and with it the array, so the kept
// address is stale afterwards: this entry point does not survive a reset.
static ks_status scratch_address(int dev, uint32_t** out) {
  if (dev < 0 || dev >= NA_MAX_DEVICES) return KS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return KS_ERR_CUDA;
    g_scratch_addr[dev] = (uint32_t*)p;
  }
  *out = g_scratch_addr[dev];
  return KS_OK;
}

}  // namespace ks

extern "C" ks_status ks_step_n_noalloc(ks_ensemble* e, uint32_t n_steps, void* stream) {
  using namespace ks;
  if (!e) return KS_ERR_INVALID_ARG;
  const uint32_t* order = nullptr;
  const uint4* items = nullptr;
  uint32_t nm = 0, ni = 0;
  ks_status s = internal_batched_schedule(e, &order, &items, &nm, &ni);
  if (s != KS_OK) return s;
  if (nm > KS_NOALLOC_MAX_MARKETS || ni > KS_NOALLOC_MAX_MARKETS) return KS_ERR_UNSUPPORTED;
  if (n_steps == 0) return KS_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return KS_ERR_CUDA;
  if (dev != internal_device(e)) return KS_ERR_INVALID_ARG;
  uint32_t* base = nullptr;
  s = scratch_address(dev, &base);
  if (s != KS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // Each call copies the schedule from the ensemble's host vectors, which
  // ks_set_batch_plan may free later: a captured graph would replay reads of
  // that memory, so a capturing stream is refused.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return KS_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return KS_ERR_UNSUPPORTED;
  // the array keeps the previous call's contents: the ticket must start at
  // zero (the step-counter kernel re-arms it after every launch; clearing it
  // here too covers a launch that failed before re-arming it)
  if (cudaMemsetAsync(base, 0, 64 * sizeof(uint32_t), st) != cudaSuccess) return KS_ERR_CUDA;
  if (cudaMemcpyAsync(base + NA_ORDER, order, (size_t)nm * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return KS_ERR_CUDA;
  if (cudaMemcpyAsync(base + NA_ITEMS, items, (size_t)ni * 16, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return KS_ERR_CUDA;
  BatchArgs b;
  b.order = base + NA_ORDER;
  b.items = reinterpret_cast<const uint4*>(base + NA_ITEMS);
  b.n_items = ni;
  b.ticket = base;
  return internal_launch_batched(e, n_steps, b, st);
}
