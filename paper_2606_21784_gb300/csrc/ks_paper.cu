// ks_paper.cu -- the paper's own agent model (Sec. III-C NOISE / MOMENTUM /
// MAKER agents around the mid price, SplitMix64 draws of Sec. III-G) on a
// tick-aggregated book, as a persistent kernel and its C ABI (ks_paper_*).
//
// A group of GT threads (a whole CTA, or one warp of a 128-thread CTA for
// markets of up to 32 x AK agents; AK up to 32) runs one market at a time for all n steps
// of a call, markets dealt round-robin.  Thread t of the group owns agents
// [t*AK, t*AK+AK) (their classes packed in one register) and ticks
// [t*LT, t*LT+LT) of the book in shared memory (BUY[p] at word 2p, SELL[p]
// at 2p+1).  Step s, between four group barriers:
//   orders    every agent draws two SplitMix64 words and adds its order to the
//             book with a shared reduction                   (Alg. 1, Phase 3)
//   B1..B3    suffix / prefix scans by warp shuffles, lowest / highest
//             maximiser of min(D, S) by redux.sync and shared atomicMax
//                                                            (Eq. 1-2, Phase 4)
//   residual  tick owners compute the unfilled part of the step's orders (the
//             resting book), fold its best bid / best ask into shared keys for
//             the next step's mid price, and clear their ticks; at the last
//             step of the call they write the resting book out  (Phase 5)
//   B5        next step's mid visible, book empty
// Global memory is read once and written once per market and call.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <type_traits>

#include "kineticsim.h"
#include "ks_market.cuh"

namespace ks {

void internal_set_error(const char* msg);

constexpr int PAPER_NOISE = 0;
constexpr int PAPER_MOMENTUM = 1;
constexpr int PAPER_MAKER = 2;
constexpr int PMI32 = 8;  // last, mid2, trades, last_v
constexpr int PMI64 = 4;  // sum_p, sum_v, hash, window origin

struct PaperParams {
  uint32_t M, market_base;
  int32_t L, A;
  uint64_t seed;
  int32_t noise2;     // 2 * noise_halfwidth
  uint32_t eta4;      // 4 * noise_halfwidth
  uint32_t p_mkt;
  uint32_t qmax;
  int32_t maker2;     // 2 * maker_half_spread
  uint32_t mom_pct, maker_pct;
  int32_t tie_rule;
  int32_t window;     // 1: sliding window with recentring
  uint32_t trace_markets, trace_steps;
  int32_t* bid;       // [M][L]
  int32_t* ask;       // [M][L]
  int32_t* mi32;      // [M][PMI32]
  int64_t* mi64;      // [M][PMI64]
  int32_t* trace;     // [trace_markets][trace_steps][2]
  uint32_t* err;
  uint64_t* step;
};

// ---- SplitMix64 (Steele, Lea, Flood, OOPSLA 2014; mixer as printed in Sec. III-G) ----
constexpr uint64_t SM64_GAMMA = 0x9E3779B97F4A7C15ull;
constexpr uint64_t SM64_GID = SM64_GAMMA << 35;  // counter step of one agent id (gid * 2^35)

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// round(x / 2^33) of x = hi * 2^32 + lo (hi signed) to the nearest integer,
// ties to even: the quotient is hi >> 1 (floor) and the remainder
// (hi & 1) * 2^32 + lo is compared with half the divisor, 2^32.
__device__ __forceinline__ int round_even_2p33(int32_t hi, uint32_t lo) {
  const int q = hi >> 1;
  const bool up = (hi & 1) && (lo != 0u || (q & 1));
  return q + (up ? 1 : 0);
}

// ---- one agent's decision (Sec. III-C), shared by the persistent and the naive kernel ----
// abase = seed + gamma * gid * 2^35 is the agent's counter origin.

// Class of the agent: percentile of channel 2 at step 0 (MAKER below maker_pct,
// then MOMENTUM below maker_pct + mom_pct, else NOISE).
__device__ __forceinline__ uint32_t paper_class(const PaperParams& P, uint64_t abase) {
  const uint32_t w = (uint32_t)(sm64_mix(abase + 2ull * SM64_GAMMA) >> 32);
  const uint32_t pct = __umulhi(w, 100u);
  return pct < P.maker_pct ? PAPER_MAKER : (pct < P.maker_pct + P.mom_pct ? PAPER_MOMENTUM : PAPER_NOISE);
}

struct PaperOrder {
  int tick, q;
  uint32_t sell;
};

// Order of agent a (class c) at step s: c0 = abase + gamma * 8s is the counter
// of channel 0 (channel 1 follows it); mid2 = 2 * mid, ret the sign of the mid's
// last change.
__device__ __forceinline__ PaperOrder paper_order(const PaperParams& P, uint64_t c0, uint32_t c, uint32_t a,
                                                  uint32_t s, int mid2, int ret) {
  const uint64_t u0 = sm64_mix(c0);
  const uint64_t u1 = sm64_mix(c0 + SM64_GAMMA);
  const uint32_t w_mkt = (uint32_t)(u0 >> 32), w_coin = (uint32_t)u0;
  const uint32_t w_price = (uint32_t)(u1 >> 32), w_qty = (uint32_t)u1;
  const bool maker = c == PAPER_MAKER;
  const bool mom = c == PAPER_MOMENTUM;
  const uint32_t coin = w_coin >> 31;
  PaperOrder o;
  o.sell = maker ? (a + s) & 1u : ((mom && ret != 0) ? (uint32_t)(ret < 0) : coin);
  const bool mkt = !maker && w_mkt < P.p_mkt;
  // round(mid + eta) (noise), round(mid +/- 1) (momentum), round(mid -/+ D) (maker):
  // the value times 2^33 is base2 * 2^32 + scale * w
  const int base2 = maker ? mid2 + (o.sell ? P.maker2 : -P.maker2) : (mom ? mid2 + (o.sell ? -2 : 2) : mid2 - P.noise2);
  const uint32_t scale = (maker || mom) ? 0u : P.eta4;
  const uint64_t prod = (uint64_t)scale * (uint64_t)w_price;
  const int rounded = round_even_2p33(base2 + (int32_t)(prod >> 32), (uint32_t)prod);
  o.tick = mkt ? (o.sell ? 0 : P.L - 1) : min(max(rounded, 0), P.L - 1);
  o.q = 1 + (int)__umulhi(w_qty, P.qmax);
  return o;
}

// Sliding window (Sec. III-A): when the mid (mid2 = 2 mid, window ticks) is
// more than L/4 from the window's centre, the window moves by an even number
// of ticks k = 2 floor((mid2 - 2 (L/2)) / 4) so that the mid is back on the
// centre (even, so ties-to-even rounding is the same in window and absolute
// ticks).  Returns k (0: no move).
__device__ __forceinline__ int window_shift(int mid2, int L) {
  const int dev = mid2 - 2 * (L / 2);
  if (dev <= L / 2 && dev >= -(L / 2)) return 0;
  return 2 * ((dev - (dev & 3)) / 4);  // dev & 3 = dev mod 4 in two's complement
}

// Shared memory of one market.
struct PaperSmem {
  int32_t* book;                 // 2 * book_len(L) words
  unsigned long long* kx;        // [2][4] argmax keys per parity
  int64_t* wbase;                // window origin (absolute tick of window tick 0); thread 0 only
  int32_t* bbk;                  // [2][2] best bid (max) / best ask (min) of the resting book per parity
  int32_t* wD;                   // [32]
  int32_t* wS;                   // [32]
};

__host__ __device__ inline size_t paper_smem_bytes(int L) {
  return (size_t)4 * 2 * book_len(L) + 8 * 8 + 8 + 4 * 4 + 4 * 64;
}

__device__ __forceinline__ PaperSmem paper_carve(unsigned char* raw, int L) {
  PaperSmem s;
  s.book = reinterpret_cast<int32_t*>(raw);
  s.kx = reinterpret_cast<unsigned long long*>(raw + (size_t)4 * 2 * book_len(L));
  s.wbase = reinterpret_cast<int64_t*>(s.kx + 8);
  s.bbk = reinterpret_cast<int32_t*>(s.wbase + 1);
  s.wD = s.bbk + 4;
  s.wS = s.wD + 32;
  return s;
}

// Groups narrower than a warp (GT = 16: two markets per warp) run their warp
// collectives on their own lane segment: mask, width and leader below.
template <int GT>
__device__ __forceinline__ unsigned seg_mask() {
  if constexpr (GT >= 32) {
    return 0xffffffffu;
  } else {
    return ((1u << GT) - 1u) << ((threadIdx.x & 31u) & ~(unsigned)(GT - 1));
  }
}

// Barrier of a market's group: the lane segment, the warp, or a named barrier.
template <int GT>
__device__ __forceinline__ void psync(int bar) {
  if constexpr (GT < 32) {
    __syncwarp(seg_mask<GT>());
  } else {
    gsync<GT>(bar);
  }
}

// Local best bid (highest tick with resting buy quantity) and best ask
// (lowest tick with resting sell quantity) folded into the shared keys by
// each warp's (or segment's) leader.
template <int GT>
__device__ __forceinline__ void fold_best(int32_t* keys, int bb, int ba) {
  constexpr int W = GT < 32 ? GT : 32;
  const unsigned fm = seg_mask<GT>();
  const int wbb = (int)__reduce_max_sync(fm, (unsigned)(bb + 1)) - 1;
  const int wba = (int)__reduce_min_sync(fm, (unsigned)ba);
  if ((threadIdx.x & (W - 1)) == 0) {
    atomicMax(keys + 0, wbb);
    atomicMin(keys + 1, wba);
  }
}

template <int NT, int AK, int LTC>
__device__ __forceinline__ void paper_market(const PaperParams& P, uint32_t m, uint32_t s0, uint32_t n_steps,
                                             const PaperSmem& sm, int t, int bar) {
  const int lane = t & 31;  // lane within the group's warp or segment
  const int wid = t >> 5;
  constexpr int W = NT < 32 ? NT : 32;  // lanes that scan and reduce together
  const unsigned FM = seg_mask<NT>();
  const int L = P.L, A = P.A;
  const int LT = (L + NT - 1) / NT;
  const int p0 = t * LT;
  const bool mine = p0 < L;
  int32_t* book = sm.book;
  const uint32_t book_s = (uint32_t)__cvta_generic_to_shared(book);
  const size_t moff = (size_t)m * (size_t)L;

  // ---- the resting book's best bid / ask give the first step's mid --------------------
  if (t < 4) sm.bbk[t] = (t & 1) ? L : -1;  // both parities: best bid -1, best ask L
  for (int i = t; i < 2 * book_len(L); i += NT) book[i] = 0;
  if (t < 8) sm.kx[t] = 0ull;
  psync<NT>(bar);
  {
    int bb = -1, ba = L;
    for (int i = 0; i < LT; ++i) {
      const int p = p0 + i;
      if (p < L) {
        if (P.bid[moff + p] > 0) bb = p;
        if (P.ask[moff + p] > 0 && ba == L) ba = p;
      }
    }
    fold_best<NT>(sm.bbk, bb, ba);
  }
  const int32_t* mi = P.mi32 + (size_t)m * PMI32;
  int last = mi[0];
  int pmid2 = mi[1];
  int trades = mi[2];
  int lastv = mi[3];
  const int64_t* m64 = P.mi64 + (size_t)m * PMI64;
  int64_t sump = m64[0], sumv = m64[1];
  uint64_t hash = (uint64_t)m64[2];
  if (t == 0) *sm.wbase = m64[3];

  // ---- agent classes (channel 2 of step 0), two bits per agent ----------------------------
  const uint64_t gid0 = (uint64_t)(P.market_base + m) * (uint64_t)A + (uint64_t)(t * AK);
  const uint64_t abase = P.seed + SM64_GID * gid0;  // + gamma * (8 s + c) + SM64_GID * k
  using ClassWord = typename std::conditional<(AK > 16), uint64_t, uint32_t>::type;
  ClassWord cls = 0;
#pragma unroll
  for (int k = 0; k < AK; ++k) cls |= (ClassWord)paper_class(P, abase + SM64_GID * (uint64_t)k) << (2 * k);
  const bool tie1 = P.tie_rule == KS_TIE_MIN_IMBALANCE;
  const bool traced = m < P.trace_markets;
  psync<NT>(bar);

  for (uint32_t j = 0; j < n_steps; ++j) {
    const uint32_t s = s0 + j;
    const int32_t* keys = sm.bbk + 2 * (j & 1);
    const int bb = keys[0], ba = keys[1];
    int mid2 = (bb >= 0 && ba < L) ? bb + ba : 2 * last;
    const int ret = (mid2 > pmid2) - (mid2 < pmid2);
    if (P.window) {
      const int k = window_shift(mid2, L);  // uniform over the group
      mid2 -= 2 * k;
      last -= k;
      if (t == 0) *sm.wbase += k;
    }

    // ---- orders of step s ---------------------------------------------------------------
    const uint64_t sbase = abase + SM64_GAMMA * (8ull * (uint64_t)s);
#pragma unroll
    for (int k = 0; k < AK; ++k) {
      const int a = t * AK + k;
      const PaperOrder o = paper_order(P, sbase + SM64_GID * (uint64_t)k, (uint32_t)(cls >> (2 * k)) & 3u,
                                       (uint32_t)a, s, mid2, ret);
      red_add_if(book_s + 4u * (uint32_t)(2 * o.tick + (int)o.sell), o.q, a < A);
    }
    psync<NT>(bar);  // B1: the step's orders are in the book

    // ---- clearing (Eq. 1-2) ---------------------------------------------------------------
    constexpr int R = LTC > 0 ? LTC : 1;
    int bv[R], sv[R];
    int sumB = 0, sumS = 0;
    if constexpr (LTC > 0) {
      if (mine) {
        ld_pairs<LTC>(book + 2 * p0, bv, sv);
      } else {
#pragma unroll
        for (int i = 0; i < LTC; ++i) bv[i] = sv[i] = 0;
      }
#pragma unroll
      for (int i = 0; i < LTC; ++i) {
        sumB += bv[i];
        sumS += sv[i];
      }
    } else {
      for (int i = 0; i < LT; ++i)
        if (p0 + i < L) {
          sumB += book[2 * (p0 + i)];
          sumS += book[2 * (p0 + i) + 1];
        }
    }
    int sufB = sumB, preS = sumS;
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
      const int vb = __shfl_down_sync(FM, sufB, d, W);
      const int vs = __shfl_up_sync(FM, preS, d, W);
      if (lane + d < W) sufB += vb;
      if (lane >= d) preS += vs;
    }
    if (lane == 0) sm.wD[wid] = sufB;
    if (lane == W - 1) sm.wS[wid] = preS;
    unsigned long long* kx = sm.kx + 4 * (j & 1);
    psync<NT>(bar);  // B2
    const int offD = (int)__reduce_add_sync(FM, (lane < NT / 32 && lane > wid) ? (unsigned)sm.wD[lane] : 0u);
    const int offS = (int)__reduce_add_sync(FM, (lane < wid) ? (unsigned)sm.wS[lane] : 0u);
    const int D0 = offD + sufB;
    const int Sb0 = offS + preS - sumS;
    {
      int D = D0, Sb = Sb0;
      int bestV = -1, lo = 4095, hi = 0;
      unsigned long long kT = 0ull;
      auto visit = [&](int p, int b, int sq) {
        const int S = Sb + sq;
        const int v = min(D, S);
        if (v > bestV) { bestV = v; lo = p; }
        if (v >= bestV) hi = p;
        if (tie1) {
          const int imb = min(abs(D - S), (1 << 22) - 1);
          const unsigned long long tk = ((unsigned long long)(uint32_t)v << 34) |
                                        ((unsigned long long)((1 << 22) - 1 - imb) << 12) | (4095u - p);
          kT = tk > kT ? tk : kT;
        }
        D -= b;
        Sb = S;
      };
      if constexpr (LTC > 0) {
        if (mine) {
#pragma unroll
          for (int i = 0; i < LTC; ++i) visit(p0 + i, bv[i], sv[i]);
        }
      } else {
        for (int i = 0; i < LT; ++i)
          if (p0 + i < L) visit(p0 + i, book[2 * (p0 + i)], book[2 * (p0 + i) + 1]);
      }
      const int vw = (int)__reduce_max_sync(FM, (unsigned)max(bestV, 0));
      const bool top = bestV == vw;
      const uint32_t low = __reduce_min_sync(FM, top ? (unsigned)lo : 4095u);
      const uint32_t high = __reduce_max_sync(FM, top ? (unsigned)hi : 0u);
      if (tie1) {
#pragma unroll
        for (int d = W / 2; d > 0; d >>= 1) {
          const unsigned long long o = __shfl_xor_sync(FM, kT, d, W);
          kT = o > kT ? o : kT;
        }
      }
      if (lane == 0) {
        atomicMax(kx + 0, ((unsigned long long)(uint32_t)vw << 12) | (4095u - low));
        atomicMax(kx + 1, ((unsigned long long)(uint32_t)vw << 12) | high);
        if (tie1) atomicMax(kx + 2, kT);
      }
    }
    psync<NT>(bar);  // B3
    const unsigned long long kLo = kx[0], kHi = kx[1];
    const int vstar = (int)(kLo >> 12);
    const int p_lo = 4095 - (int)(kLo & 4095u);
    const int p_hi = (int)(kHi & 4095u);
    const int pstar = tie1 ? 4095 - (int)(kx[2] & 4095u) : p_lo;
    const bool trade = vstar > 0;
    if (t < 4) sm.kx[4 * ((j + 1) & 1) + t] = 0ull;  // the other parity's keys for the next step
    int32_t* nkeys = sm.bbk + 2 * ((j + 1) & 1);       // (reset by the previous step, see below)
    const bool final_step = j + 1 == n_steps;

    // ---- resting book: the unfilled part of the step's orders (Phase 5) --------------------
    {
      int D = D0, Sb = Sb0;
      int nbb = -1, nba = L;
      auto rest = [&](int p, int b, int sq) {
        int nb = b, ns = sq;
        if (trade) {
          const int rb = vstar - (D - b);  // units filled at the marginal buy tick
          const int rs = vstar - Sb;       // units filled at the marginal sell tick
          nb = p > p_hi ? 0 : (p == p_hi ? b - rb : b);
          ns = p < p_lo ? 0 : (p == p_lo ? sq - rs : sq);
        }
        D -= b;
        Sb += sq;
        if (nb > 0) nbb = p;
        if (ns > 0 && nba == L) nba = p;
        if (final_step) {
          P.bid[moff + p] = nb;
          P.ask[moff + p] = ns;
        }
      };
      if constexpr (LTC > 0) {
        if (mine) {
          int z[R];
#pragma unroll
          for (int i = 0; i < LTC; ++i) {
            rest(p0 + i, bv[i], sv[i]);
            z[i] = 0;
          }
          st_pairs<LTC>(book + 2 * p0, z, z);
        }
      } else {
        for (int i = 0; i < LT; ++i) {
          const int p = p0 + i;
          if (p < L) {
            rest(p, book[2 * p], book[2 * p + 1]);
            book[2 * p] = 0;
            book[2 * p + 1] = 0;
          }
        }
      }
      fold_best<NT>(nkeys, nbb, nba);
    }
    if (t == 0) {
      // keys of the step after next start empty (this step read them already)
      sm.bbk[2 * (j & 1)] = -1;
      sm.bbk[2 * (j & 1) + 1] = L;
    }
    // ---- market scalars ---------------------------------------------------------------------
    if (trade) last = pstar;
    pmid2 = mid2;
    if (t == 0) {
      const int64_t base = *sm.wbase;
      const int pt = trade ? (int)(base + pstar) : -1;  // absolute p*
      if (trade) {
        sump += base + pstar;
        trades += 1;
      }
      sumv += vstar;
      lastv = vstar;
      hash = trace_mix(hash, s, pt, vstar);
      if (traced && s < P.trace_steps) {
        int32_t* tr = P.trace + ((size_t)m * P.trace_steps + s) * 2;
        tr[0] = P.window ? (int)(base + last) : pt;  // window: the absolute last price, carried
        tr[1] = vstar;
      }
    }
    psync<NT>(bar);  // B5: next mid keys complete, book empty
  }
  if (t == 0) {
    int32_t* mo = P.mi32 + (size_t)m * PMI32;
    mo[0] = last;
    mo[1] = pmid2;
    mo[2] = trades;
    mo[3] = lastv;
    int64_t* mo64 = P.mi64 + (size_t)m * PMI64;
    mo64[0] = sump;
    mo64[1] = sumv;
    mo64[2] = (int64_t)hash;
    mo64[3] = *sm.wbase;
  }
  psync<NT>(bar);  // shared memory is reused by the group's next market
}

// Shared memory per group, 16-byte aligned.
__host__ __device__ inline size_t paper_group_bytes(int L) { return (paper_smem_bytes(L) + 15) & ~(size_t)15; }

// CTA of NT threads in groups of GT (NT / GT markets in parallel; GT = 16 and
// GT = 32 groups synchronise with __syncwarp on their lanes, larger ones with
// named barriers).
// MINB > 1: compiled for at least MINB resident CTAs per SM (a register cap).
template <int NT, int GT, int AK, int MINB>
__global__ void __launch_bounds__(NT, MINB) paper_kernel(PaperParams P, uint32_t n_steps) {
  static_assert(GT == 16 || GT == 32 || GT == NT, "groups are half a warp, one warp or the whole CTA");
  constexpr int G = NT / GT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const uint32_t s0 = (uint32_t)(*P.step);
  const int g = (int)threadIdx.x / GT;
  const PaperSmem sm = paper_carve(smem_raw + (size_t)g * paper_group_bytes(P.L), P.L);
  const int LT = (P.L + GT - 1) / GT;
  const int LTsel = ((LT == 1 || LT == 2 || LT == 4 || LT == 8) && (P.L % LT == 0)) ? LT : 0;
  if (P.A > GT * AK) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(P.err, ERR_SHAPE);
    return;
  }
  const int t = (int)threadIdx.x % GT;
  for (uint32_t m = blockIdx.x * G + g; m < P.M; m += gridDim.x * G) {
    switch (LTsel) {
      case 1: paper_market<GT, AK, 1>(P, m, s0, n_steps, sm, t, 0); break;
      case 2: paper_market<GT, AK, 2>(P, m, s0, n_steps, sm, t, 0); break;
      case 4: paper_market<GT, AK, 4>(P, m, s0, n_steps, sm, t, 0); break;
      case 8: paper_market<GT, AK, 8>(P, m, s0, n_steps, sm, t, 0); break;
      default: paper_market<GT, AK, 0>(P, m, s0, n_steps, sm, t, 0); break;
    }
  }
}

__global__ void paper_init_kernel(PaperParams P) {
  for (uint32_t m = blockIdx.x; m < P.M; m += gridDim.x) {
    for (int p = threadIdx.x; p < P.L; p += blockDim.x) {
      P.bid[(size_t)m * P.L + p] = 0;
      P.ask[(size_t)m * P.L + p] = 0;
    }
    if (threadIdx.x == 0) {
      int32_t* mi = P.mi32 + (size_t)m * PMI32;
      mi[0] = P.L / 2;
      mi[1] = 2 * (P.L / 2);
      for (int i = 2; i < PMI32; ++i) mi[i] = 0;
      int64_t* m64 = P.mi64 + (size_t)m * PMI64;
      for (int i = 0; i < PMI64; ++i) m64[i] = 0;
    }
  }
}

__global__ void paper_step_bump(uint64_t* step, uint32_t n) { *step += n; }

// Roofline probe: the two SplitMix64 mixes of one agent-step (channels 0 and 1)
// in a loop with nothing else, one agent per thread and iteration.
__global__ void __launch_bounds__(256) probe_sm64(uint32_t iters, uint64_t* sink) {
  uint64_t c = SM64_GID * (uint64_t)(blockIdx.x * 256u + threadIdx.x);
  uint64_t acc = 0;
  for (uint32_t it = 0; it < iters; ++it) {
    const uint64_t u0 = sm64_mix(c), u1 = sm64_mix(c + SM64_GAMMA);
    acc ^= u0 ^ (u1 << 1);
    c += 8ull * SM64_GAMMA;
  }
  sink[(size_t)blockIdx.x * 256u + threadIdx.x] = acc;
}

// Launches probe_sm64 (256-thread blocks); returns the mixes it computes.
double launch_probe_sm64(uint32_t blocks, uint32_t iters, uint64_t* sink, cudaStream_t st) {
  probe_sm64<<<blocks, 256, 0, st>>>(iters, sink);
  return 2.0 * (double)blocks * 256.0 * (double)iters;
}

// ---- the naive engine: one thread per market, one launch per step (Sec. III-F, Sec. IV-I) ----
// Same model, decisions and draws as paper_kernel (paper_class / paper_order),
// without its two design choices: the book stays in global memory (each step
// reads the resting rows for the best bid / ask, aggregates the step's orders
// into the same rows and writes the residual back: Theta(L) loads and stores
// per market and step) and clearing is one serial sweep per market (scans and
// argmax in one upward pass from the total demand, then the residual pass).
constexpr int PAPER_NAIVE_THREADS = 128;

__global__ void __launch_bounds__(PAPER_NAIVE_THREADS) paper_naive_kernel(PaperParams P) {
  const uint32_t m = blockIdx.x * PAPER_NAIVE_THREADS + threadIdx.x;
  if (m >= P.M) return;
  const uint32_t s = (uint32_t)(*P.step);
  const int L = P.L, A = P.A;
  int32_t* bid = P.bid + (size_t)m * (size_t)L;
  int32_t* ask = P.ask + (size_t)m * (size_t)L;
  int32_t* mi = P.mi32 + (size_t)m * PMI32;
  int64_t* m64 = P.mi64 + (size_t)m * PMI64;

  // mid of the resting book; the rows are then reused for the step's orders
  int bb = -1, ba = L;
  for (int p = 0; p < L; ++p) {
    if (bid[p] > 0) bb = p;
    if (ask[p] > 0 && ba == L) ba = p;
    bid[p] = 0;
    ask[p] = 0;
  }
  int last0 = mi[0];
  int mid2 = (bb >= 0 && ba < L) ? bb + ba : 2 * last0;
  const int pmid2 = mi[1];
  const int ret = (mid2 > pmid2) - (mid2 < pmid2);
  int64_t base = m64[3];
  if (P.window) {
    const int k = window_shift(mid2, L);
    base += k;
    mid2 -= 2 * k;
    last0 -= k;
  }

  // orders of step s, agent by agent
  const uint64_t mbase = P.seed + SM64_GID * ((uint64_t)(P.market_base + m) * (uint64_t)A);
  const uint64_t sofs = SM64_GAMMA * (8ull * (uint64_t)s);
  int Dtot = 0;
  for (int a = 0; a < A; ++a) {
    const uint64_t abase = mbase + SM64_GID * (uint64_t)a;
    const PaperOrder o = paper_order(P, abase + sofs, paper_class(P, abase), (uint32_t)a, s, mid2, ret);
    if (o.sell) {
      ask[o.tick] += o.q;
    } else {
      bid[o.tick] += o.q;
      Dtot += o.q;
    }
  }

  // clearing (Eq. 1-2): D = D_cum[p] and S = S_cum[p] in one upward sweep
  const bool tie1 = P.tie_rule == KS_TIE_MIN_IMBALANCE;
  int D = Dtot, Sb = 0;
  int bestV = -1, lo = 0, hi = 0;
  int v1 = -1, imb1 = 0, p1 = 0;
  for (int p = 0; p < L; ++p) {
    const int S = Sb + ask[p];
    const int v = min(D, S);
    if (v > bestV) {
      bestV = v;
      lo = p;
    }
    if (v >= bestV) hi = p;
    if (tie1) {
      const int imb = min(abs(D - S), (1 << 22) - 1);
      if (v > v1 || (v == v1 && imb < imb1)) {
        v1 = v;
        imb1 = imb;
        p1 = p;
      }
    }
    D -= bid[p];
    Sb = S;
  }
  const int vstar = max(bestV, 0);
  const bool trade = vstar > 0;
  const int pstar = tie1 ? p1 : lo;

  // residual: buys fill from the top down to the highest maximiser, sells from
  // the bottom up to the lowest one (the marginal ticks, rationed)
  if (trade) {
    D = Dtot;
    Sb = 0;
    for (int p = 0; p < L; ++p) {
      const int b = bid[p], sq = ask[p];
      const int rb = vstar - (D - b);
      const int rs = vstar - Sb;
      bid[p] = p > hi ? 0 : (p == hi ? b - rb : b);
      ask[p] = p < lo ? 0 : (p == lo ? sq - rs : sq);
      D -= b;
      Sb += sq;
    }
  }

  // market scalars (prices in the trace, the sum and the hash are absolute)
  const int pt = trade ? (int)(base + pstar) : -1;
  const int last = trade ? pstar : last0;
  mi[0] = last;
  mi[1] = mid2;
  if (trade) {
    mi[2] += 1;
    m64[0] += base + pstar;
  }
  mi[3] = vstar;
  m64[1] += vstar;
  m64[2] = (int64_t)trace_mix((uint64_t)m64[2], s, pt, vstar);
  m64[3] = base;
  if (m < P.trace_markets && s < P.trace_steps) {
    int32_t* tr = P.trace + ((size_t)m * P.trace_steps + s) * 2;
    tr[0] = P.window ? (int)(base + last) : pt;
    tr[1] = vstar;
  }
}

using PaperLaunchFn = void (*)(const PaperParams&, uint32_t, int, size_t, cudaStream_t);
template <int NT, int GT, int AK, int MINB>
void paper_launch(const PaperParams& p, uint32_t n, int grid, size_t smem, cudaStream_t st) {
  paper_kernel<NT, GT, AK, MINB><<<grid, NT, smem, st>>>(p, n);
}

struct PaperVariant {
  int threads;  // threads per market (group); a 32-thread group shares a 128-thread CTA with three others
  int ak, min_ctas;
  int cta_threads;
  PaperLaunchFn launch;
  const void* kernel;
};
#define KS_PV(NT, GT, AK, MB)                                                                  \
  PaperVariant {                                                                               \
    GT, AK, MB, NT, &paper_launch<NT, GT, AK, MB>, (const void*)&paper_kernel<NT, GT, AK, MB> \
  }
// (threads per market, agents per thread, 1 = compiler's register choice,
// else the register cap of that many resident CTAs; 32 x 8 at 6 spills a few words)
static const PaperVariant kPaperVariants[] = {
    KS_PV(128, 32, 1, 1),    KS_PV(128, 32, 2, 1),    KS_PV(128, 32, 4, 1),    KS_PV(128, 32, 1, 8),
    KS_PV(128, 32, 2, 8),    KS_PV(128, 32, 8, 1),    KS_PV(128, 32, 8, 6),    KS_PV(128, 32, 16, 1),
    KS_PV(128, 32, 32, 1),    KS_PV(128, 128, 1, 1),   KS_PV(128, 128, 2, 1),   KS_PV(128, 128, 4, 1),
    KS_PV(128, 128, 8, 1),   KS_PV(128, 128, 16, 1),  KS_PV(128, 128, 1, 8),   KS_PV(128, 128, 2, 8),
    KS_PV(128, 128, 4, 6),   KS_PV(128, 128, 8, 6),   KS_PV(256, 256, 1, 1),   KS_PV(256, 256, 2, 1),
    KS_PV(256, 256, 4, 1),   KS_PV(256, 256, 8, 1),   KS_PV(256, 256, 16, 1),  KS_PV(512, 512, 16, 1),
    KS_PV(1024, 1024, 16, 1), KS_PV(128, 16, 1, 1),    KS_PV(128, 16, 2, 1),    KS_PV(128, 16, 4, 1),
    KS_PV(128, 16, 2, 8),    KS_PV(128, 16, 4, 8),    KS_PV(64, 64, 4, 1),     KS_PV(64, 64, 8, 1)};
#undef KS_PV

}  // namespace ks

using namespace ks;

struct ks_paper_ensemble {
  PaperParams p;
  uint32_t M;
  int L, A;
  const PaperVariant* var;
  int grid;
  size_t smem;
  int num_sms;
  int device;
};

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct PaperLayout {
  size_t bid, ask, mi32, mi64, trace, ctrl, total;
};

PaperLayout paper_layout(const ks_paper_config* c) {
  PaperLayout l;
  size_t o = 0;
  const size_t ML = (size_t)c->n_markets * (size_t)c->L;
  l.bid = o; o = al256(o + ML * 4);
  l.ask = o; o = al256(o + ML * 4);
  l.mi32 = o; o = al256(o + (size_t)c->n_markets * PMI32 * 4);
  l.mi64 = o; o = al256(o + (size_t)c->n_markets * PMI64 * 8);
  l.trace = o; o = al256(o + (size_t)c->trace_markets * c->trace_steps * 2 * 4);
  l.ctrl = o; o = al256(o + 64);  // err (u32) at +0, step (u64) at +8
  l.total = o;
  return l;
}

ks_status fail(ks_status s, const char* msg) {
  internal_set_error(msg);
  return s;
}

ks_status cuda_status(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  internal_set_error(buf);
  return KS_ERR_CUDA;
}

#define KSP_CUDA(call)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_status(e_, #call);  \
  } while (0)

ks_status validate(const ks_paper_config* c) {
  if (!c) return fail(KS_ERR_INVALID_ARG, "config is NULL");
  if (c->n_markets == 0) return fail(KS_ERR_INVALID_ARG, "n_markets must be >= 1");
  if (c->n_markets > (1u << 26)) return fail(KS_ERR_UNSUPPORTED, "n_markets above 2^26");
  if ((uint64_t)c->market_base + c->n_markets > 0xFFFFFFFFull)
    return fail(KS_ERR_INVALID_ARG, "market_base + n_markets above 2^32");
  if (c->L < 2 || c->L > KS_MAX_TICKS) return fail(KS_ERR_UNSUPPORTED, "L outside [2, KS_MAX_TICKS]");
  if (c->A < 0 || c->A > KS_MAX_AGENTS) return fail(KS_ERR_UNSUPPORTED, "A outside [0, KS_MAX_AGENTS]");
  if (c->qmax < 1 || c->qmax > KS_MAX_QTY) return fail(KS_ERR_INVALID_ARG, "qmax outside [1, KS_MAX_QTY]");
  if (c->noise_halfwidth < 0 || c->noise_halfwidth > c->L)
    return fail(KS_ERR_INVALID_ARG, "noise_halfwidth outside [0, L]");
  if (c->maker_half_spread < 0 || c->maker_half_spread > c->L)
    return fail(KS_ERR_INVALID_ARG, "maker_half_spread outside [0, L]");
  if (c->mom_pct + c->maker_pct > 100u) return fail(KS_ERR_INVALID_ARG, "mom_pct + maker_pct above 100");
  if (c->tie_rule != KS_TIE_LOWEST_TICK && c->tie_rule != KS_TIE_MIN_IMBALANCE)
    return fail(KS_ERR_INVALID_ARG, "unknown tie_rule");
  if (c->window != 0 && c->window != 1) return fail(KS_ERR_INVALID_ARG, "window must be 0 or 1");
  // per-step volume: A orders of at most KS_MAX_QTY must fit int32 (and the 22-bit imbalance key)
  if ((int64_t)c->A * c->qmax >= (1ll << 31)) return fail(KS_ERR_UNSUPPORTED, "A * qmax above 2^31");
  return KS_OK;
}

ks_status apply_launch(ks_paper_ensemble* e, int threads, int ak, int min_ctas) {
  const PaperVariant* v = nullptr;
  for (const auto& x : kPaperVariants)
    if (x.threads == threads && x.ak == ak && x.min_ctas == std::max(min_ctas, 1)) v = &x;
  if (!v) return fail(KS_ERR_INVALID_ARG, "no paper-agent kernel for this (threads, agents_per_thread, min_ctas)");
  if ((int64_t)threads * ak < e->A) return fail(KS_ERR_INVALID_ARG, "threads * agents_per_thread below A");
  const int G = v->cta_threads / v->threads;  // markets per CTA
  const size_t smem = (size_t)G * paper_group_bytes(e->L);
  if (smem > 200 * 1024) return fail(KS_ERR_UNSUPPORTED, "launch shape needs more shared memory than a CTA has");
  KSP_CUDA(cudaFuncSetAttribute(v->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  KSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v->kernel, v->cta_threads, smem));
  if (occ < 1) return fail(KS_ERR_UNSUPPORTED, "launch shape does not fit on an SM");
  e->var = v;
  e->smem = smem;
  e->grid = (int)std::min<int64_t>(((int64_t)e->M + G - 1) / G, (int64_t)occ * e->num_sms);
  return KS_OK;
}

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

extern "C" {

ks_status ks_paper_workspace_size(const ks_paper_config* cfg, size_t* bytes) {
  if (!bytes) return fail(KS_ERR_INVALID_ARG, "bytes is NULL");
  ks_status s = validate(cfg);
  if (s != KS_OK) return s;
  *bytes = paper_layout(cfg).total;
  return KS_OK;
}

ks_status ks_paper_create(const ks_paper_config* cfg, void* workspace, size_t ws_bytes, void* stream,
                          ks_paper_ensemble** out) {
  if (!out) return fail(KS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  ks_status s = validate(cfg);
  if (s != KS_OK) return s;
  if (!workspace) return fail(KS_ERR_INVALID_ARG, "workspace is NULL");
  if (((uintptr_t)workspace & 255u) != 0) return fail(KS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  const PaperLayout lay = paper_layout(cfg);
  if (ws_bytes < lay.total) return fail(KS_ERR_WORKSPACE_TOO_SMALL, "workspace below ks_paper_workspace_size");
  ks_paper_ensemble* e = new ks_paper_ensemble();
  unsigned char* ws = (unsigned char*)workspace;
  PaperParams& p = e->p;
  memset(&p, 0, sizeof(p));
  p.M = cfg->n_markets;
  p.market_base = cfg->market_base;
  p.L = cfg->L;
  p.A = cfg->A;
  p.seed = cfg->seed;
  p.noise2 = 2 * cfg->noise_halfwidth;
  p.eta4 = 4u * (uint32_t)cfg->noise_halfwidth;
  p.p_mkt = cfg->p_mkt_q32;
  p.qmax = (uint32_t)cfg->qmax;
  p.maker2 = 2 * cfg->maker_half_spread;
  p.mom_pct = cfg->mom_pct;
  p.maker_pct = cfg->maker_pct;
  p.tie_rule = cfg->tie_rule;
  p.window = cfg->window;
  p.trace_markets = std::min(cfg->trace_markets, cfg->n_markets);
  p.trace_steps = cfg->trace_markets ? cfg->trace_steps : 0;
  p.bid = (int32_t*)(ws + lay.bid);
  p.ask = (int32_t*)(ws + lay.ask);
  p.mi32 = (int32_t*)(ws + lay.mi32);
  p.mi64 = (int64_t*)(ws + lay.mi64);
  p.trace = (int32_t*)(ws + lay.trace);
  p.err = (uint32_t*)(ws + lay.ctrl);
  p.step = (uint64_t*)(ws + lay.ctrl + 8);
  e->M = cfg->n_markets;
  e->L = cfg->L;
  e->A = cfg->A;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t ce;
  if ((ce = cudaGetDevice(&e->device)) != cudaSuccess ||
      (ce = cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device)) != cudaSuccess ||
      (ce = cudaMemsetAsync(ws + lay.ctrl, 0, 64, st)) != cudaSuccess ||
      (ce = cudaMemsetAsync(ws + lay.trace, 0xFF, lay.ctrl - lay.trace, st)) != cudaSuccess) {
    delete e;
    return cuda_status(ce, "ks_paper_create");
  }
  paper_init_kernel<<<std::min<uint32_t>(e->M, 4096u), 128, 0, st>>>(p);
  if ((ce = cudaGetLastError()) != cudaSuccess) {
    delete e;
    return cuda_status(ce, "paper_init_kernel");
  }
  // default shape (measured on GB300 at L = 128 with 8192 markets): half a
  // warp per market up to 32 agents, a warp up to 256 agents, else 128
  // threads per market with up to 16 agents each, under the register caps
  // that won; two warps per market when only 513 to 2048 markets share the GPU
  int nt = cfg->A <= 256 ? 32 : 128;
  while (nt < 1024 && (int64_t)nt * 16 < cfg->A) nt *= 2;
  int ak = std::min(16, next_pow2(std::max(1, (cfg->A + nt - 1) / nt)));
  int mc = nt == 32 ? (ak == 8 ? 6 : 1) : ((nt == 128 && ak <= 2) ? 8 : ((nt == 128 && ak <= 8) ? 6 : 1));
  if (cfg->A <= 32) {
    nt = 16;
    ak = 2;
    mc = 8;
  } else if (cfg->A <= 512 && cfg->n_markets > 512 && cfg->n_markets <= 2048) {
    // too few markets to fill the GPU one warp each: two warps per market
    nt = 64;
    ak = cfg->A <= 256 ? 4 : 8;
    mc = 1;
  }
  s = apply_launch(e, nt, ak, mc);
  if (s != KS_OK) {
    delete e;
    return s;
  }
  *out = e;
  return KS_OK;
}

ks_status ks_paper_step_n(ks_paper_ensemble* e, uint32_t n_steps, void* stream) {
  if (!e) return fail(KS_ERR_INVALID_ARG, "ensemble is NULL");
  if (n_steps == 0) return KS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  e->var->launch(e->p, n_steps, e->grid, e->smem, st);
  KSP_CUDA(cudaGetLastError());
  paper_step_bump<<<1, 1, 0, st>>>(e->p.step, n_steps);
  KSP_CUDA(cudaGetLastError());
  return KS_OK;
}

ks_status ks_paper_step_n_naive(ks_paper_ensemble* e, uint32_t n_steps, void* stream) {
  if (!e) return fail(KS_ERR_INVALID_ARG, "ensemble is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = (int)((e->p.M + PAPER_NAIVE_THREADS - 1) / PAPER_NAIVE_THREADS);
  for (uint32_t i = 0; i < n_steps; ++i) {
    paper_naive_kernel<<<grid, PAPER_NAIVE_THREADS, 0, st>>>(e->p);
    KSP_CUDA(cudaGetLastError());
    paper_step_bump<<<1, 1, 0, st>>>(e->p.step, 1);
    KSP_CUDA(cudaGetLastError());
  }
  return KS_OK;
}

ks_status ks_paper_read_state(ks_paper_ensemble* e, const ks_paper_state_view* v, void* stream) {
  if (!e || !v) return fail(KS_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const PaperParams& p = e->p;
  const size_t ML = (size_t)e->M * (size_t)e->L;
  if (v->bid) KSP_CUDA(cudaMemcpyAsync(v->bid, p.bid, ML * 4, cudaMemcpyDefault, st));
  if (v->ask) KSP_CUDA(cudaMemcpyAsync(v->ask, p.ask, ML * 4, cudaMemcpyDefault, st));
  struct F {
    void* view;
    const void* dev;
    size_t pitch, width;
  } fs[] = {
      {v->last_tick, p.mi32 + 0, PMI32 * 4, 4}, {v->mid2, p.mi32 + 1, PMI32 * 4, 4},
      {v->trades, p.mi32 + 2, PMI32 * 4, 4},    {v->last_volume, p.mi32 + 3, PMI32 * 4, 4},
      {v->sum_price, p.mi64 + 0, PMI64 * 8, 8}, {v->sum_volume, p.mi64 + 1, PMI64 * 8, 8},
      {v->trace_hash, p.mi64 + 2, PMI64 * 8, 8}, {v->window_base, p.mi64 + 3, PMI64 * 8, 8},
  };
  for (auto& f : fs)
    if (f.view) KSP_CUDA(cudaMemcpy2DAsync(f.view, f.width, f.dev, f.pitch, f.width, e->M, cudaMemcpyDefault, st));
  if (v->step) KSP_CUDA(cudaMemcpyAsync(v->step, p.step, 8, cudaMemcpyDefault, st));
  if (v->trace)
    KSP_CUDA(cudaMemcpyAsync(v->trace, p.trace, (size_t)p.trace_markets * p.trace_steps * 2 * 4, cudaMemcpyDefault,
                             st));
  KSP_CUDA(cudaStreamSynchronize(st));
  return KS_OK;
}

ks_status ks_paper_set_launch(ks_paper_ensemble* e, int32_t threads, int32_t agents_per_thread, int32_t min_ctas) {
  if (!e) return fail(KS_ERR_INVALID_ARG, "ensemble is NULL");
  return apply_launch(e, threads, agents_per_thread, min_ctas);
}

ks_status ks_paper_get_launch(const ks_paper_ensemble* e, int32_t* threads, int32_t* agents_per_thread,
                              int32_t* min_ctas) {
  if (!e || !threads || !agents_per_thread || !min_ctas) return fail(KS_ERR_INVALID_ARG, "NULL argument");
  *threads = e->var->threads;
  *agents_per_thread = e->var->ak;
  *min_ctas = e->var->min_ctas;
  return KS_OK;
}

ks_status ks_paper_sync(ks_paper_ensemble* e, void* stream, uint32_t timeout_ms) {
  if (!e) return fail(KS_ERR_INVALID_ARG, "ensemble is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ev;
  KSP_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t ce = cudaEventRecord(ev, st);
  if (ce != cudaSuccess) {
    cudaEventDestroy(ev);
    return cuda_status(ce, "cudaEventRecord");
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    ce = cudaEventQuery(ev);
    if (ce == cudaSuccess) break;
    if (ce != cudaErrorNotReady) {
      cudaEventDestroy(ev);
      return cuda_status(ce, "cudaEventQuery");
    }
    if (timeout_ms) {
      const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
      if (ms.count() >= (long long)timeout_ms) {
        cudaEventDestroy(ev);
        return fail(KS_ERR_TIMEOUT, "ks_paper_sync deadline passed before the stream finished");
      }
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  uint32_t word = 0;
  KSP_CUDA(cudaMemcpyAsync(&word, e->p.err, 4, cudaMemcpyDeviceToHost, st));
  KSP_CUDA(cudaStreamSynchronize(st));
  if (word) {
    char buf[64];
    snprintf(buf, sizeof(buf), "device error word 0x%x", word);
    internal_set_error(buf);
    return KS_ERR_DEVICE_FAULT;
  }
  return KS_OK;
}

ks_status ks_paper_destroy(ks_paper_ensemble* e) {
  delete e;
  return KS_OK;
}

}  // extern "C"
