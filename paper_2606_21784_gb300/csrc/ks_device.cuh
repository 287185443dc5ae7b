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
constexpr uint32_t W_ST = W_SIDE | (W_TICK << W_TICK_SHIFT);  // side and tick bits

// The book interleaves the two sides per tick: BUY[p] at word 2p, SELL[p]
// at 2p + 1.  The index of an order word is then its bits 8-20 as they stand.
__device__ __forceinline__ int bidx(uint32_t sell, uint32_t tick) { return (int)(2u * tick + sell); }
__device__ __forceinline__ uint32_t w_bidx(uint32_t w) { return (w >> 8) & 0x1FFFu; }

// Ticks of a market's book in shared memory, rounded to 16 so that a thread
// can load the (BUY, SELL) pairs of its contiguous ticks with vector accesses
// (contiguous vector accesses across a warp are free of bank conflicts).
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

// The same block with precomputed round keys (rk as in DevParams::rk).
__device__ __forceinline__ uint4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) philox_round(c0, c1, c2, c3, rk[2 * r], rk[2 * r + 1]);
  return make_uint4(c0, c1, c2, c3);
}

// Per-step draws use counter (step, agent, market, 0).  Within one step and
// market only the agent word varies, so the parts of rounds 1-3 that do not
// depend on it are computed once (StepKey) and each agent finishes the block
// with 16 instead of 20 wide multiplies.  The result equals philox() exactly.
// Round keys come from rk (the kernel parameters: constant-bank operands).
struct StepKey {
  uint32_t c0;    // round-1 word 0 without the agent term
  uint32_t x3k;   // round-1 word 3 xor round-2 key 1
  uint32_t y1k;   // round-2 word 1 xor round-3 key 0
  uint32_t hAk;   // round-3 hi(A) xor round-3 key 1
  uint32_t z3;    // round-3 word 3
};

__device__ __forceinline__ StepKey step_key(uint32_t step, uint32_t market, uint32_t stream, const uint32_t* rk) {
  StepKey s;
  // round 1 (key k): A = MA*step, B = MB*market
  uint32_t hA, lA, hB, lB;
  mulhilo(PH_MA, step, hA, lA);
  mulhilo(PH_MB, market, hB, lB);
  uint32_t x1 = lB;
  uint32_t x2 = hA ^ stream ^ rk[1];
  uint32_t x3 = lA;
  s.c0 = hB ^ rk[0];  // x0 = c0 ^ agent
  // round 2 (key k + W): B = MB*x2 is agent independent
  uint32_t hB2, lB2;
  mulhilo(PH_MB, x2, hB2, lB2);
  uint32_t y0 = hB2 ^ x1 ^ rk[2];
  uint32_t y1 = lB2;
  s.x3k = x3 ^ rk[3];
  // round 3 (key k + 2W): A = MA*y0 is agent independent
  uint32_t hA3, lA3;
  mulhilo(PH_MA, y0, hA3, lA3);
  s.y1k = y1 ^ rk[4];
  s.hAk = hA3 ^ rk[5];
  s.z3 = lA3;
  return s;
}

// x0 = s.c0 ^ agent (an agent index a0 + k with a0 a multiple of a power of
// two above k is s.c0 ^ a0 ^ k: one xor per agent).
__device__ __forceinline__ uint4 step_draw_x0(const StepKey& s, uint32_t x0, const uint32_t* rk) {
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
  for (int r = 3; r < 10; ++r) philox_round(z0, z1, z2, z3, rk[2 * r], rk[2 * r + 1]);
  return make_uint4(z0, z1, z2, z3);
}

// floor(w * n / 2^32)
__device__ __forceinline__ uint32_t range_u32(uint32_t w, uint32_t n) { return __umulhi(w, n); }

// Rule parameters of the ensemble (derived from ks_config once per market).
struct RuleConsts {
  int32_t zi_off;
  uint32_t zi_n;     // 2*zi_off + 1
  uint32_t zi_qmax;
  uint32_t mom_n;    // mom_offset_max + 1
  uint32_t mr_n;     // mr_offset_max + 1
  uint32_t rb_qmax;
};

// 256-bit global accesses (sm_100 and later): one lane moves a whole 32-byte
// sector, so a warp's strided state accesses write no partial sectors.  The
// address must be 32-byte aligned.
__device__ __forceinline__ void ld_b32x8(const void* p, uint32_t (&v)[8]) {
  asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void st_b32x8(void* p, const uint32_t (&v)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]),
               "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void ld_b64x4(const void* p, int64_t (&v)[4]) {
  asm volatile("ld.global.v4.b64 {%0,%1,%2,%3}, [%4];" : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_b64x4(void* p, const int64_t (&v)[4]) {
  asm volatile("st.global.v4.b64 [%0], {%1,%2,%3,%4};" ::"l"(p), "l"(v[0]), "l"(v[1]), "l"(v[2]), "l"(v[3]) : "memory");
}

// Asynchronous L2 prefetch of [p, p + bytes) (cp.async.bulk.prefetch.L2),
// widened to 16-byte bounds.  The callers' ranges lie in workspace regions that
// are 256-byte aligned and padded to 256 bytes, so the widened range stays in
// the region.  Nothing waits for it.
__device__ __forceinline__ void l2_prefetch(const void* p, size_t bytes) {
  uint64_t g;
  asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(p));
  const uint64_t lo = g & ~15ull;
  const uint64_t n = ((g + bytes + 15ull) & ~15ull) - lo;
  if (n > 0 && n < (1ull << 31))
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)n) : "memory");
}

// book[i] += v where pred holds, as one predicated shared-memory reduction
// (no branch around it).
__device__ __forceinline__ void red_add_if(uint32_t saddr, int v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q red.shared.add.s32 [%0], %1;\n\t}" ::"r"(saddr),
      "r"(v), "r"((int)pred));
}

// ---------------------------------------------------------------------------
// Rule-based decision of an agent without a working order, from the draw
// words w = (w0 cancel, w1 side, w2 offset, w3 quantity) of its Philox block:
//   zero intelligence: sell iff w1 >= 2^31; tick = last - zi_off +
//     floor(w2 (2 zi_off + 1) / 2^32); qty = 1 + floor(w3 zi_qmax / 2^32);
//   momentum: side = sign of the lookback return of the last clearing tick
//     (buy if up, sell if down, the w1 coin if flat); mean reversion: side
//     toward the market's fundamental tick (the coin at the fundamental);
//     both order o = floor(w2 (omax + 1) / 2^32) ticks through the last tick
//     (a buy at last + o, a sell at last - o), qty 1 + floor(w3 rb_qmax / 2^32);
// ticks clamped to [0, L).  Within a step everything but the draw words is
// the same for all agents of a class, so the step's constants sit in a
// 4-row table in shared memory indexed by the class bits of the order word
// (class 3, never assigned, behaves as mean reversion).  Row fields: sell
// iff bit 31 of (w1 & coin_mask) | forced_sell; o = floor(w2 n / 2^32);
// tick = clamp(base + sgn o) with sgn = -1 if w1 & sgn_mask, else sgn_fix;
// qty = 1 + floor(w3 qmax / 2^32).
// ---------------------------------------------------------------------------
struct ClassRule {
  uint32_t n, qmax, coin_mask, forced_sell;
  uint32_t sgn_mask;
  int32_t sgn_fix, base, pad;
};

// Row c of the table for a step whose last clearing tick is `last`;
// side_mom / side_mr: 0 buy, 1 sell, -1 undecided.
__device__ __forceinline__ ClassRule class_rule(int c, int last, int side_mom, int side_mr, const RuleConsts& rc) {
  ClassRule r;
  r.pad = 0;
  if (c == KS_CLASS_ZI) {
    r.n = rc.zi_n;
    r.qmax = rc.zi_qmax;
    r.coin_mask = 0x80000000u;
    r.forced_sell = 0u;
    r.sgn_mask = 0u;
    r.sgn_fix = 1;
    r.base = last - rc.zi_off;
  } else {
    const int side = c == KS_CLASS_MOM ? side_mom : side_mr;
    r.n = c == KS_CLASS_MOM ? rc.mom_n : rc.mr_n;
    r.qmax = rc.rb_qmax;
    r.base = last;
    if (side < 0) {
      r.coin_mask = 0x80000000u;
      r.forced_sell = 0u;
      r.sgn_mask = 0x80000000u;
      r.sgn_fix = 1;
    } else {
      r.coin_mask = 0u;
      r.forced_sell = (uint32_t)side << 31;
      r.sgn_mask = 0u;
      r.sgn_fix = side ? -1 : 1;
    }
  }
  return r;
}

// New order word of an agent (static bits of `slot` kept) from its table row.
__device__ __forceinline__ uint32_t decide_tab(uint32_t slot, uint4 w, const ClassRule* tab, int L) {
  const uint4 a = *reinterpret_cast<const uint4*>(tab + w_class(slot));
  const uint4 b = *(reinterpret_cast<const uint4*>(tab + w_class(slot)) + 1);
  const uint32_t sell31 = (w.y & a.z) | a.w;
  const int o = (int)__umulhi(w.z, a.x);
  const int sgn = (w.y & b.x) ? -1 : (int)b.y;
  const int tick = min(max((int)b.z + sgn * o, 0), L - 1);
  const uint32_t qty = 1u + __umulhi(w.w, a.y);
  return (slot & W_STATIC) | qty | (sell31 >> 23) | ((uint32_t)tick << W_TICK_SHIFT);
}

// The same decision from eight rows indexed by (class, side coin), the coin
// being bit 31 of w1: row 2c + coin holds {n, qmax, base, sgn} with the
// side and the offset's sign already resolved, and sell[2c + coin] the side
// bit of the order word.  Equal to decide_tab for every input.
__device__ __forceinline__ void decision_row(uint4* rows, uint32_t* sell, int r, int last, int side_mom, int side_mr,
                                             const RuleConsts& rc) {
  const ClassRule cr = class_rule(r >> 1, last, side_mom, side_mr, rc);
  const uint32_t coin = (uint32_t)(r & 1) << 31;
  const int sgn = (coin & cr.sgn_mask) ? -1 : cr.sgn_fix;
  rows[r] = make_uint4(cr.n, cr.qmax, (uint32_t)cr.base, (uint32_t)sgn);
  sell[r] = ((coin & cr.coin_mask) | cr.forced_sell) ? W_SIDE : 0u;
}

__device__ __forceinline__ uint32_t decide_rows(uint32_t slot, uint4 w, const uint4* rows, const uint32_t* sell, int L) {
  const uint32_t idx = ((slot >> (W_CLASS_SHIFT - 1)) & 6u) | (w.y >> 31);
  const uint4 r = rows[idx];
  const int o = (int)__umulhi(w.z, r.x);
  const int tick = min(max((int)r.z + (int)r.w * o, 0), L - 1);
  const uint32_t qty = 1u + __umulhi(w.w, r.y);
  return (slot & W_STATIC) | qty | sell[idx] | ((uint32_t)tick << W_TICK_SHIFT);
}

// SplitMix64 finaliser (Sec. III-G) folding the per-step clearing trace.
__device__ __forceinline__ uint64_t trace_mix(uint64_t h, uint32_t step, int32_t pstar, int32_t vol) {
  uint64_t z = h ^ (((uint64_t)(uint32_t)pstar << 32) | (uint64_t)(uint32_t)vol) ^
               ((uint64_t)step * 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace ks
