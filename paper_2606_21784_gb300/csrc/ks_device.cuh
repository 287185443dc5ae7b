// ks_device.cuh -- device primitives of the persistent call-auction kernels:
// Philox4x32-10 draws, agent decision rules, order-word packing.
#pragma once

#include <stdint.h>

#include "ks_internal.h"

namespace ks {

// ---------------------------------------------------------------------------
// Order word (see kineticsim.h): qty 0-7, side 8, tick 9-20, class 21-22, mlp 23.
// ---------------------------------------------------------------------------
constexpr uint32_t W_QTY = 0xFFu;
constexpr uint32_t W_SIDE = 1u << 8;
constexpr int W_TICK_SHIFT = 9;
constexpr uint32_t W_TICK = 0xFFFu;
constexpr int W_CLASS_SHIFT = 21;
constexpr uint32_t W_MLP = 1u << 23;
constexpr uint32_t W_STATIC = (3u << W_CLASS_SHIFT) | W_MLP;  // survives an empty slot

__device__ __forceinline__ uint32_t w_qty(uint32_t w) { return w & W_QTY; }
__device__ __forceinline__ uint32_t w_sell(uint32_t w) { return (w >> 8) & 1u; }
__device__ __forceinline__ uint32_t w_tick(uint32_t w) { return (w >> W_TICK_SHIFT) & W_TICK; }
__device__ __forceinline__ uint32_t w_class(uint32_t w) { return (w >> W_CLASS_SHIFT) & 3u; }

// Length of one half (BUY or SELL) of a market's book in shared memory:
// rounded to 16 ticks so that both halves start 64-byte aligned and a thread
// can load its contiguous ticks with vector accesses (contiguous vector
// accesses across a warp are free of bank conflicts).
__host__ __device__ __forceinline__ int book_len(int L) { return (L + 15) & ~15; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Round: with products
// A = 0xD2511F53 * x0 and B = 0xCD9E8D57 * x2 (64-bit), the next counter is
// (hi(B) ^ x1 ^ k0, lo(B), hi(A) ^ x3 ^ k1, lo(A)); the key advances by the
// Weyl constants (0x9E3779B9, 0xBB67AE85) before every round but the first.
// ---------------------------------------------------------------------------
constexpr uint32_t PH_MA = 0xD2511F53u;
constexpr uint32_t PH_MB = 0xCD9E8D57u;
constexpr uint32_t PH_WA = 0x9E3779B9u;
constexpr uint32_t PH_WB = 0xBB67AE85u;

__device__ __forceinline__ void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

__device__ __forceinline__ void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                             uint32_t k0, uint32_t k1) {
  uint32_t hA, lA, hB, lB;
  mulhilo(PH_MA, x0, hA, lA);
  mulhilo(PH_MB, x2, hB, lB);
  uint32_t y0 = hB ^ x1 ^ k0;
  uint32_t y2 = hA ^ x3 ^ k1;
  x0 = y0;
  x1 = lB;
  x2 = y2;
  x3 = lA;
}

// Generic block for any counter (used off the hot loop).
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(c0, c1, c2, c3, k0 + (uint32_t)r * PH_WA, k1 + (uint32_t)r * PH_WB);
  }
  return make_uint4(c0, c1, c2, c3);
}

// Per-step draws use counter (step, agent, market, 0).  Within one step and
// market only the agent word varies, so the parts of rounds 1-3 that do not
// depend on it are computed once (StepKey) and each agent finishes the block
// with 16 instead of 20 wide multiplies.  The result equals philox() exactly.
struct StepKey {
  uint32_t c0;    // round-1 word 0 without the agent term
  uint32_t x3k;   // round-1 word 3 xor round-2 key 1
  uint32_t y1k;   // round-2 word 1 xor round-3 key 0
  uint32_t hAk;   // round-3 hi(A) xor round-3 key 1
  uint32_t z3;    // round-3 word 3
  uint32_t k0, k1;
};

__device__ __forceinline__ StepKey step_key(uint32_t step, uint32_t market, uint32_t stream, uint32_t k0,
                                            uint32_t k1) {
  StepKey s;
  // round 1 (key k): A = MA*step, B = MB*market
  uint32_t hA, lA, hB, lB;
  mulhilo(PH_MA, step, hA, lA);
  mulhilo(PH_MB, market, hB, lB);
  uint32_t x1 = lB;
  uint32_t x2 = hA ^ stream ^ k1;
  uint32_t x3 = lA;
  s.c0 = hB ^ k0;  // x0 = c0 ^ agent
  // round 2 (key k + W): B = MB*x2 is agent independent
  uint32_t hB2, lB2;
  mulhilo(PH_MB, x2, hB2, lB2);
  uint32_t y0 = hB2 ^ x1 ^ (k0 + PH_WA);
  uint32_t y1 = lB2;
  s.x3k = x3 ^ (k1 + PH_WB);
  // round 3 (key k + 2W): A = MA*y0 is agent independent
  uint32_t hA3, lA3;
  mulhilo(PH_MA, y0, hA3, lA3);
  s.y1k = y1 ^ (k0 + 2u * PH_WA);
  s.hAk = hA3 ^ (k1 + 2u * PH_WB);
  s.z3 = lA3;
  s.k0 = k0;
  s.k1 = k1;
  return s;
}

__device__ __forceinline__ uint4 step_draw(const StepKey& s, uint32_t agent) {
  uint32_t x0 = s.c0 ^ agent;
  // round 2, agent-dependent half: A = MA*x0
  uint32_t hA2, lA2;
  mulhilo(PH_MA, x0, hA2, lA2);
  uint32_t y2 = hA2 ^ s.x3k;
  uint32_t y3 = lA2;
  // round 3, agent-dependent half: B = MB*y2
  uint32_t hB3, lB3;
  mulhilo(PH_MB, y2, hB3, lB3);
  uint32_t z0 = hB3 ^ s.y1k;
  uint32_t z1 = lB3;
  uint32_t z2 = s.hAk ^ y3;
  uint32_t z3 = s.z3;
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    philox_round(z0, z1, z2, z3, s.k0 + (uint32_t)r * PH_WA, s.k1 + (uint32_t)r * PH_WB);
  }
  return make_uint4(z0, z1, z2, z3);
}

// floor(w * n / 2^32)
__device__ __forceinline__ uint32_t range_u32(uint32_t w, uint32_t n) { return __umulhi(w, n); }

// ---------------------------------------------------------------------------
// Rule-based decision of an agent without a working order.
// side_mom / side_mr: 0 buy, 1 sell, -1 undecided (use the draw's side bit).
// Returns the new order word (static bits of `slot` kept).
// ---------------------------------------------------------------------------
struct RuleConsts {
  int32_t zi_off;
  uint32_t zi_n;     // 2*zi_off + 1
  uint32_t zi_qmax;
  uint32_t mom_n;    // mom_offset_max + 1
  uint32_t mr_n;     // mr_offset_max + 1
  uint32_t rb_qmax;
};

__device__ __forceinline__ uint32_t decide_rule(uint32_t slot, uint4 w, int last, int side_mom, int side_mr,
                                                int L, const RuleConsts& rc) {
  uint32_t cls = w_class(slot);
  uint32_t coin = w.y >> 31;  // 0 buy (w1 < 2^31), 1 sell
  bool zi = cls == KS_CLASS_ZI;
  int sd_rule = cls == KS_CLASS_MOM ? side_mom : side_mr;
  uint32_t sell = zi ? coin : (sd_rule < 0 ? coin : (uint32_t)sd_rule);
  uint32_t n = zi ? rc.zi_n : (cls == KS_CLASS_MOM ? rc.mom_n : rc.mr_n);
  int o = (int)range_u32(w.z, n);
  int off = zi ? o - rc.zi_off : (sell ? -o : o);
  int tick = min(max(last + off, 0), L - 1);
  uint32_t qmax = zi ? rc.zi_qmax : rc.rb_qmax;
  uint32_t qty = 1u + range_u32(w.w, qmax);
  return (slot & W_STATIC) | qty | (sell << 8) | ((uint32_t)tick << W_TICK_SHIFT);
}

// SplitMix64 finaliser (Sec. III-F) folding the per-step clearing trace.
__device__ __forceinline__ uint64_t trace_mix(uint64_t h, uint32_t step, int32_t pstar, int32_t vol) {
  uint64_t z = h ^ (((uint64_t)(uint32_t)pstar << 32) | (uint64_t)(uint32_t)vol) ^
               ((uint64_t)step * 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace ks
