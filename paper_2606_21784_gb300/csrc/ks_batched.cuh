// ks_batched.cuh -- one persistent launch over markets of uneven (L, A).
//
// The host sorts markets into (L, A) buckets, gives each bucket a group shape
// (GT threads per market, AK agents per thread) and packs the markets of a
// bucket into work items of up to G = min(NT / GT, shared-memory fit) markets.
// Items are ordered longest first (LPT).  Every CTA repeatedly takes the next
// item from a global ticket counter, splits itself into G groups that run one
// market each (named barriers per group, __syncwarp for one-warp groups), and
// moves on when all its groups are done.
#pragma once

#include "ks_market.cuh"

namespace ks {

struct BatchArgs {
  const uint32_t* order;  // market indices grouped by item
  const uint4* items;     // {first, count, variant, Lcap}
  uint32_t n_items;
  uint32_t* ticket;       // next item (reset to 0 after every launch)
};

template <int NT, int GT, int AK>
__device__ __forceinline__ void run_item(const DevParams& P, const BatchArgs& B, uint4 d, uint32_t s0, uint32_t n,
                                         unsigned char* raw) {
  static_assert(GT == 32 || GT == NT || NT / GT <= 15, "named barrier ids 1..15");
  constexpr int G = NT / GT;
  const int g = (int)threadIdx.x / GT;
  if (g < G && g < (int)d.y) {
    constexpr int BUDGET = thread_reg_budget(NT, 1);  // the batched kernels' launch bounds
    constexpr bool REGACC = accounts_in_registers(BUDGET, AK, false);
    size_t o[8];
    const size_t gsz = group_smem_layout(BUDGET, GT, AK, (int)d.w, false, o);
    const Smem sm = carve<GT, AK, false, !REGACC>(raw + (size_t)g * gsz, (int)d.w);
    const int bar = (GT == NT) ? 0 : 1 + g;
    run_market<GT, AK, false, false, REGACC, true>(P, B.order[d.x + g], s0, n, sm, (int)threadIdx.x % GT, bar, (int)d.w);
  }
}

// Policy-capable variant: each warpgroup of a group also owns an mbarrier,
// MLP_TMEM_COLS TMEM columns of the CTA (its tile accumulator and
// activations) and a named barrier, and evaluates policy tiles.
template <int NT, int GT, int AK>
__device__ __forceinline__ void run_item_mlp(const DevParams& P, const BatchArgs& B, uint4 d, uint32_t s0, uint32_t n,
                                             unsigned char* raw, const MlpCta& mc) {
  static_assert(GT >= 128 && GT % 128 == 0, "policy groups are whole warpgroups");
  constexpr int G = NT / GT;
  const int g = (int)threadIdx.x / GT;
  if (g < G && g < (int)d.y) {
    size_t o[8];
    const size_t gsz = group_smem_layout(thread_reg_budget(NT, 1), GT, AK, (int)d.w, true, o);
    const int ntw = GT / 128;  // every warpgroup of the group evaluates policy tiles
    unsigned char* graw = raw + (size_t)g * gsz;
    const Smem sm = carve<GT, AK, true, true>(graw, (int)d.w);
    const int bar = (GT == NT) ? 0 : 1 + g;
    const int wl = ((int)threadIdx.x % GT) / 128;  // warpgroup in the group
    const int wc = (int)threadIdx.x / 128;         // warpgroup in the CTA
    MlpWG mw;
    mw.wg = wl;
    mw.nwg = ntw;
    mw.bar = &mc.bars[wc];
    mw.tmem = *mc.tslot + (uint32_t)(wc * MLP_TMEM_COLS);
    mw.bar_id = (GT == 128) ? bar : 8 + wc;
    mw.phase = 0;
    mw.abort = false;
    run_market<GT, AK, false, true, false, true>(P, B.order[d.x + g], s0, n, sm, (int)threadIdx.x % GT, bar, (int)d.w, &mw,
                                    mc.sw);
  }
}

#define KS_BATCH_MLP_VARIANTS_512(X) \
  X(0, 128, 4) X(1, 128, 8) X(2, 128, 16) X(3, 256, 8) X(4, 256, 16) X(5, 512, 8) X(6, 512, 16) X(7, 512, 32)

template <int NT>
__device__ __forceinline__ void dispatch_item_mlp(const DevParams& P, const BatchArgs& B, uint4 d, uint32_t s0, uint32_t n,
                                  unsigned char* raw, const MlpCta& mc);

template <int NT>
__global__ void __launch_bounds__(NT, 1) batched_mlp_kernel(DevParams P, uint32_t n_steps, BatchArgs B) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint32_t s_item;
  const uint32_t s0 = (uint32_t)(*P.step);
  static_assert(NT / 128 <= MLP_MAX_TILE_WGS, "one TMEM share per warpgroup");
  const MlpCta mc = mlp_cta_carve(smem_raw, (uint32_t)(NT / 128) * MLP_TMEM_COLS);
  mlp_cta_setup(mc, P.mlp);
  unsigned char* raw = smem_raw + mlp_cta_bytes();
  for (;;) {
    __syncthreads();  // the previous item is finished and s_item has been read
    if (threadIdx.x == 0) {
      s_item = atomicAdd(B.ticket, 1u);
      // every group starts the item at mbarrier phase 0 (no MMA is in flight here)
      for (int i = 0; i < MLP_MAX_GROUPS; ++i) mbar_init(&mc.bars[i], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= B.n_items) break;
    dispatch_item_mlp<NT>(P, B, B.items[it], s0, n_steps, raw, mc);
  }
  mlp_cta_teardown(mc);
}

// (variant id, GT, AK) lists; the host mirrors them in ks_batched_variants().
#define KS_BATCH_VARIANTS_1024(X)                                                                          \
  X(0, 32, 1) X(1, 32, 2) X(2, 32, 4) X(3, 32, 8) X(4, 128, 2) X(5, 128, 4) X(6, 128, 8) X(7, 256, 4) \
  X(8, 256, 8) X(9, 256, 16) X(10, 512, 8) X(11, 512, 16) X(12, 1024, 8) X(13, 1024, 16)
#define KS_BATCH_VARIANTS_512(X)                                                                        \
  X(0, 32, 1) X(1, 32, 2) X(2, 32, 4) X(3, 32, 8) X(4, 64, 2) X(5, 64, 4) X(6, 64, 8) X(7, 128, 4) \
  X(8, 128, 8) X(9, 256, 8) X(10, 256, 16) X(11, 512, 8) X(12, 512, 16) X(13, 512, 32)

template <int NT>
__device__ __forceinline__ void dispatch_item(const DevParams& P, const BatchArgs& B, uint4 d, uint32_t s0, uint32_t n,
                              unsigned char* raw);

template <int NT>
__global__ void __launch_bounds__(NT, 1) batched_kernel(DevParams P, uint32_t n_steps, BatchArgs B) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint32_t s_item;
  const uint32_t s0 = (uint32_t)(*P.step);
  for (;;) {
    __syncthreads();  // the previous item is finished and s_item has been read
    if (threadIdx.x == 0) s_item = atomicAdd(B.ticket, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= B.n_items) break;
    dispatch_item<NT>(P, B, B.items[it], s0, n_steps, smem_raw);
  }
}

}  // namespace ks
