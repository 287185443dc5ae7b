// ks_cda.cu -- continuous double auction over the main model's agents (see
// kineticsim.h, ks_cda_*): one warp per market, the book in shared memory.
//
// The book of a market is a FIFO of resting agents per (side, tick): a
// circular list through per-agent next indices whose last agent is kept per
// (side, tick) and points at the first; plus one bitmap of nonempty ticks per
// side, so the best bid and ask are found with a few word scans.  Per step
// the warp's lanes draw the Philox blocks, cancel and decide for 32 agents at
// a time (the per-step cost that the call auction also has); lane 0 then
// removes the cancelled orders and matches the new orders one by one in agent
// order, which continuous trading makes sequential.  The serial matching waits on shared-memory latency, so a
// market keeps only 6 bytes per agent and 4 per tick on chip and many markets
// share an SM: lane 0 adds every fill to the inventory and cash in global
// memory with reductions (no kernel reads them back), and an agent that
// cancels draws its new order again after the cancellations instead of
// keeping it.  Only the next indices persist in global memory (-1 after the
// last agent of a FIFO); the circular links, the last agents and the bitmaps
// are rebuilt when a market is loaded.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <thread>

#include "kineticsim.h"
#include "ks_device.cuh"
#include "ks_internal.h"

namespace ks {

void internal_set_error(const char* msg);
cudaError_t internal_init_state(const DevParams& p, int grid, cudaStream_t st);

namespace {

struct CdaParams {
  uint32_t M, market_base;
  int32_t L, A;
  uint32_t rk[20];
  uint32_t cancel_thr;
  RuleConsts rc;
  int32_t mom_lb;
  uint32_t trace_markets, trace_steps;
  uint32_t* ord;
  int32_t* inv;
  int64_t* cash;
  int32_t* nxt;
  int32_t* mi32;  // [M][MI32_STRIDE] as the main ensemble
  int64_t* mi64;  // [M][MI64_STRIDE]; MI_SUMP holds the traded value
  int32_t* trace;
  uint32_t* err;
  const uint64_t* step;
};

// Shared memory of one market (one warp), 16-byte aligned regions.
struct CdaSmem {
  uint32_t* ord;   // [A] order words; a deciding agent's new order until it is matched
  int16_t* nxt;    // [A] next agent in the circular FIFO; -1 without a resting order
  int16_t* tail;   // [2][L] last agent per (side, tick), -1 if empty; its next is the first
  uint32_t* bits;  // [2][NW] nonempty ticks per side
  uint32_t* cbits; // [ceil(A / 32)] cancelled this step (while loading: agents with a predecessor)
  uint32_t* dbits; // [ceil(A / 32)] deciding this step
  ClassRule* ctab; // [4]
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline int cda_words(int L) { return (L + 31) / 32; }

__host__ __device__ inline size_t cda_smem_layout(int A, int L, size_t* o) {
  size_t off = 0;
  const size_t a = (size_t)(A > 0 ? A : 1), nwa = (a + 31) / 32;
  o[0] = off; off = al16(off + 4 * a);                               // ord
  o[1] = off; off = al16(off + 2 * a);                               // nxt
  o[2] = off; off = al16(off + 2 * 2 * (size_t)L);                   // tail
  o[3] = off; off = al16(off + 4 * 2 * (size_t)cda_words(L));        // bits
  o[4] = off; off = al16(off + 4 * nwa);                             // cbits
  o[5] = off; off = al16(off + 4 * nwa);                             // dbits
  o[6] = off; off = al16(off + 4 * sizeof(ClassRule));               // ctab
  return off;
}

__device__ inline CdaSmem cda_carve(unsigned char* raw, int A, int L) {
  size_t o[7];
  cda_smem_layout(A, L, o);
  CdaSmem s;
  s.ord = reinterpret_cast<uint32_t*>(raw + o[0]);
  s.nxt = reinterpret_cast<int16_t*>(raw + o[1]);
  s.tail = reinterpret_cast<int16_t*>(raw + o[2]);
  s.bits = reinterpret_cast<uint32_t*>(raw + o[3]);
  s.cbits = reinterpret_cast<uint32_t*>(raw + o[4]);
  s.dbits = reinterpret_cast<uint32_t*>(raw + o[5]);
  s.ctab = reinterpret_cast<ClassRule*>(raw + o[6]);
  return s;
}

// Lowest nonempty tick >= from in the bitmap `b` of NW words, -1 if none.
__device__ inline int cda_scan_up(const uint32_t* b, int NW, int from, int L) {
  if (from >= L) return -1;
  if (from < 0) from = 0;
  int w = from >> 5;
  uint32_t word = b[w] & (0xFFFFFFFFu << (from & 31));
  for (;;) {
    if (word) return (w << 5) + __ffs(word) - 1;
    if (++w >= NW) return -1;
    word = b[w];
  }
}

// Highest nonempty tick <= from, -1 if none.
__device__ inline int cda_scan_down(const uint32_t* b, int from) {
  if (from < 0) return -1;
  int w = from >> 5;
  const int r = from & 31;
  uint32_t word = b[w] & (r == 31 ? 0xFFFFFFFFu : ((1u << (r + 1)) - 1u));
  for (;;) {
    if (word) return (w << 5) + 31 - __clz(word);
    if (--w < 0) return -1;
    word = b[w];
  }
}

// Book bookkeeping of lane 0: best bid (highest nonempty buy tick) and best
// ask (lowest nonempty sell tick), -1 when a side is empty.
struct CdaBest {
  int bid, ask;
};

// The FIFO of (SIDE, tick) has become empty: clear its bit and move the side's
// best price past it.
template <int SIDE>
__device__ __forceinline__ void cda_emptied(const CdaSmem& sm, int L, int NW, int tick, CdaBest& best) {
  uint32_t* b = sm.bits + SIDE * NW;
  b[tick >> 5] &= ~(1u << (tick & 31));
  if (SIDE == 0) {
    if (tick == best.bid) best.bid = cda_scan_down(b, tick - 1);
  } else {
    if (tick == best.ask) best.ask = cda_scan_up(b, NW, tick + 1, L);
  }
}

// Removes agent r, the first of the FIFO of (SIDE, tick) whose last is t.
template <int SIDE>
__device__ __forceinline__ void cda_pop(const CdaSmem& sm, int L, int NW, int r, int t, int tick, CdaBest& best) {
  const int key = SIDE * L + tick;
  if (r == t) {
    sm.tail[key] = -1;
    cda_emptied<SIDE>(sm, L, NW, tick, best);
  } else {
    sm.nxt[t] = sm.nxt[r];
  }
  sm.nxt[r] = -1;
}

// Removes agent a from anywhere in the FIFO of (SIDE, tick); its predecessor
// is found by walking the circle from the last agent (at most A + 1 links).
// False when a is not in that FIFO.
template <int SIDE>
__device__ inline bool cda_remove(const CdaSmem& sm, int L, int NW, int A, int a, int tick, CdaBest& best) {
  const int key = SIDE * L + tick;
  const int t = sm.tail[key];
  if (t < 0) return false;
  int p = t;
  for (int guard = 0; guard <= A; ++guard) {
    const int n = sm.nxt[p];
    if (n < 0) return false;
    if (n == a) {
      if (p == a) {
        sm.tail[key] = -1;
        cda_emptied<SIDE>(sm, L, NW, tick, best);
      } else {
        sm.nxt[p] = sm.nxt[a];
        if (a == t) sm.tail[key] = (int16_t)p;
      }
      sm.nxt[a] = -1;
      return true;
    }
    p = n;
  }
  return false;
}

// Appends agent a at the tail of the FIFO of (SIDE, tick).
template <int SIDE>
__device__ __forceinline__ void cda_append(const CdaSmem& sm, int L, int NW, int a, int tick, CdaBest& best) {
  const int key = SIDE * L + tick;
  const int t = sm.tail[key];
  if (t >= 0) {
    sm.nxt[a] = sm.nxt[t];
    sm.nxt[t] = (int16_t)a;
  } else {
    sm.nxt[a] = (int16_t)a;
    sm.bits[SIDE * NW + (tick >> 5)] |= 1u << (tick & 31);
    if (SIDE == 0) {
      if (tick > best.bid) best.bid = tick;
    } else {
      if (best.ask < 0 || tick < best.ask) best.ask = tick;
    }
  }
  sm.tail[key] = (int16_t)a;
}

// The new order o of agent a on side SD (0 buys, 1 sells): trades against the
// opposite side in price-time priority while its limit crosses, every fill at
// the resting order's tick, then rests its remainder.  Each fill goes to the
// resting agent's inventory and cash in global memory at once, the arriving
// agent's once for the order.  Returns the filled quantity.
template <int SD>
__device__ __forceinline__ int cda_arrive(const CdaSmem& sm, int L, int NW, int a, uint32_t o, CdaBest& best,
                                          int32_t* ginv, unsigned long long* gcash, int& last_fill, int& fills,
                                          int64_t& value, uint32_t* err) {
  constexpr int OS = 1 - SD;
  const int tk = (int)w_tick(o);
  const int16_t* ot = sm.tail + OS * L;
  int q = (int)w_qty(o);
  int dq = 0, dv = 0;  // filled quantity and traded value of the order
  while (q > 0) {
    const int px = SD == 0 ? best.ask : best.bid;
    // the limit no longer crosses, or the opposite side is empty (-1)
    if (SD == 0 ? (uint32_t)px > (uint32_t)tk : px < tk) break;
    const int t = ot[px];
    const int r = t >= 0 ? sm.nxt[t] : -1;
    if (r < 0) {  // bitmap and FIFO disagree: record it and stop matching this order
      atomicOr(err, ERR_SHAPE);
      break;
    }
    const uint32_t ro = sm.ord[r];
    const int rq = (int)w_qty(ro);
    if (rq == 0) {  // an empty order in a FIFO: record it, drop it (the loop still ends)
      atomicOr(err, ERR_SHAPE);
      cda_pop<OS>(sm, L, NW, r, t, px, best);
      continue;
    }
    const int f = min(q, rq);
    const int pf = px * f;
    atomicAdd(ginv + r, SD == 0 ? -f : f);
    atomicAdd(gcash + r, (unsigned long long)(long long)(SD == 0 ? pf : -pf));
    dq += f;
    dv += pf;
    q -= f;
    last_fill = px;
    fills += 1;
    if (f == rq) {
      cda_pop<OS>(sm, L, NW, r, t, px, best);
      sm.ord[r] = ro & W_STATIC;
    } else {
      sm.ord[r] = ro - (uint32_t)f;
    }
  }
  if (dq) {
    atomicAdd(ginv + a, SD == 0 ? dq : -dq);
    atomicAdd(gcash + a, (unsigned long long)(long long)(SD == 0 ? -dv : dv));
    value += dv;
  }
  if (q > 0) {
    sm.ord[a] = (o & ~W_QTY) | (uint32_t)q;
    cda_append<SD>(sm, L, NW, a, tk, best);
  } else {
    sm.ord[a] = o & W_STATIC;
  }
  return dq;
}

// Steps [s0, s0 + n) of market m by one warp.
__device__ void cda_market(const CdaParams& P, uint32_t m, uint32_t s0, uint32_t n, const CdaSmem& sm, int lane) {
  const int L = P.L, A = P.A, NW = cda_words(L);
  const int nwa = (A + 31) / 32;
  const int64_t aoff = (int64_t)m * A;
  const uint32_t gm = P.market_base + m;
  // ---- load and rebuild the book: links, last agents, bitmaps ------------------------------
  for (int a = lane; a < A; a += 32) {
    const uint32_t o = P.ord[aoff + a];
    const int nx = P.nxt[aoff + a];
    sm.ord[a] = o;
    sm.nxt[a] = (int16_t)(w_qty(o) != 0u && nx >= 0 && nx < A ? nx : -1);
  }
  for (int i = lane; i < 2 * L; i += 32) sm.tail[i] = -1;
  for (int i = lane; i < 2 * NW; i += 32) sm.bits[i] = 0u;
  for (int i = lane; i < nwa; i += 32) sm.cbits[i] = 0u;
  __syncwarp();
  for (int a = lane; a < A; a += 32) {
    const int nx = sm.nxt[a];
    if (nx >= 0) atomicOr(&sm.cbits[nx >> 5], 1u << (nx & 31));  // nx has a predecessor
  }
  __syncwarp();
  for (int a = lane; a < A; a += 32) {
    const uint32_t o = sm.ord[a];
    if (w_qty(o) == 0u) continue;
    const int side = (int)w_sell(o), tick = (int)w_tick(o);
    if (tick >= L) {  // written by no kernel of this library: record it, drop the order
      atomicOr(P.err, ERR_TICK);
      sm.ord[a] = o & W_STATIC;
      continue;
    }
    if (sm.nxt[a] < 0) sm.tail[side * L + tick] = (int16_t)a;
    atomicOr(&sm.bits[side * NW + (tick >> 5)], 1u << (tick & 31));
  }
  __syncwarp();
  for (int a = lane; a < A; a += 32) {  // close each FIFO: the last agent's next is the first
    const uint32_t o = sm.ord[a];
    if (w_qty(o) == 0u || (int)w_tick(o) >= L || ((sm.cbits[a >> 5] >> (a & 31)) & 1u)) continue;
    const int t = sm.tail[(int)w_sell(o) * L + (int)w_tick(o)];
    if (t >= 0) sm.nxt[t] = (int16_t)a; else atomicOr(P.err, ERR_SHAPE);
  }
  __syncwarp();
  const int32_t* mi = P.mi32 + (size_t)m * MI32_STRIDE;
  int hist[KS_HISTORY];
#pragma unroll
  for (int j = 0; j < KS_HISTORY; ++j) hist[j] = mi[MI_HIST + j];
  int last = mi[MI_LAST];
  const int fund = mi[MI_FUND];
  int fills = mi[MI_TRADES];
  int lastv = mi[MI_LASTV];
  const int64_t* mi64 = P.mi64 + (size_t)m * MI64_STRIDE;
  int64_t value = mi64[MI_SUMP];
  int64_t sumv = mi64[MI_SUMV];
  uint64_t hash = (uint64_t)mi64[MI_HASH];
  CdaBest best{-1, -1};
  if (lane == 0) {
    best.bid = cda_scan_down(sm.bits, L - 1);
    best.ask = cda_scan_up(sm.bits + NW, NW, 0, L);
  }
  const bool traced = m < P.trace_markets;
  int32_t* const ginv = P.inv + aoff;
  unsigned long long* const gcash = reinterpret_cast<unsigned long long*>(P.cash + aoff);

  for (uint32_t j = 0; j < n; ++j) {
    const uint32_t s = s0 + j;
    // ---- draws, cancellations and decisions, 32 agents at a time -----------------------
    const StepKey sk = step_key(s, gm, 0u, P.rk);
    int hlb = hist[1];  // hist[mom_lb] with compile-time indices (the history stays in registers)
#pragma unroll
    for (int i = 2; i < KS_HISTORY; ++i) hlb = (P.mom_lb == i) ? hist[i] : hlb;
    const int ret = hist[0] - hlb;
    const int side_mom = ret > 0 ? 0 : (ret < 0 ? 1 : -1);
    const int side_mr = last < fund ? 0 : (last > fund ? 1 : -1);
    if (lane < 4) sm.ctab[lane] = class_rule(lane, last, side_mom, side_mr, P.rc);
    __syncwarp();
    for (int wi = 0; wi < nwa; ++wi) {
      const int a = wi * 32 + lane;
      const bool valid = a < A;
      const uint32_t sl = valid ? sm.ord[a] : 0u;
      const uint4 w = step_draw_x0(sk, sk.c0 ^ (uint32_t)a, P.rk);
      const uint32_t q = w_qty(sl);
      const bool cancel = valid && q != 0u && w.x < P.cancel_thr;
      if (valid && q == 0u) sm.ord[a] = decide_tab(sl, w, sm.ctab, L);  // no resting order: decide in place
      const uint32_t cb = __ballot_sync(0xffffffffu, cancel);
      const uint32_t db = __ballot_sync(0xffffffffu, valid && (q == 0u || cancel));
      if (lane == 0) {
        sm.cbits[wi] = cb;
        sm.dbits[wi] = db;
      }
    }
    __syncwarp();
    // ---- lane 0: the cancellations -----------------------------------------------------------
    if (lane == 0) {
      for (int wi = 0; wi < nwa; ++wi) {
        for (uint32_t b = sm.cbits[wi]; b; b &= b - 1u) {
          const int a = wi * 32 + __ffs(b) - 1;
          const uint32_t o = sm.ord[a];
          const bool found = w_sell(o) ? cda_remove<1>(sm, L, NW, A, a, (int)w_tick(o), best)
                                       : cda_remove<0>(sm, L, NW, A, a, (int)w_tick(o), best);
          if (!found) atomicOr(P.err, ERR_SHAPE);
          sm.ord[a] = o & W_STATIC;
        }
      }
    }
    __syncwarp();
    // ---- the new orders of the agents that cancelled: the same draws again -------------------
    for (int wi = 0; wi < nwa; ++wi) {
      const uint32_t cb = sm.cbits[wi];  // the same word for every lane
      if (cb == 0u) continue;
      const int a = wi * 32 + lane;
      const uint4 w = step_draw_x0(sk, sk.c0 ^ (uint32_t)a, P.rk);
      if ((cb >> lane) & 1u) sm.ord[a] = decide_tab(sm.ord[a], w, sm.ctab, L);
    }
    __syncwarp();
    // ---- lane 0: the arrivals in agent order ---------------------------------------------------
    int last_fill = -1;
    int vol = 0;
    if (lane == 0) {
      for (int wi = 0; wi < nwa; ++wi) {
        for (uint32_t b = sm.dbits[wi]; b; b &= b - 1u) {
          const int a = wi * 32 + __ffs(b) - 1;
          const uint32_t o = sm.ord[a];
          vol += w_sell(o) ? cda_arrive<1>(sm, L, NW, a, o, best, ginv, gcash, last_fill, fills, value, P.err)
                           : cda_arrive<0>(sm, L, NW, a, o, best, ginv, gcash, last_fill, fills, value, P.err);
        }
      }
    }
    // ---- step statistics (every lane keeps the scalars) ------------------------------------
    last_fill = __shfl_sync(0xffffffffu, last_fill, 0);
    vol = __shfl_sync(0xffffffffu, vol, 0);
    fills = __shfl_sync(0xffffffffu, fills, 0);
    value = __shfl_sync(0xffffffffu, value, 0);
    if (last_fill >= 0) last = last_fill;
#pragma unroll
    for (int h = KS_HISTORY - 1; h > 0; --h) hist[h] = hist[h - 1];
    hist[0] = last;
    lastv = vol;
    sumv += vol;
    hash = trace_mix(hash, s, last_fill, vol);
    if (lane == 0 && traced && s < P.trace_steps) {
      int32_t* tr = P.trace + ((size_t)m * P.trace_steps + s) * 2;
      tr[0] = last_fill;
      tr[1] = vol;
    }
    __syncwarp();
  }
  // ---- store (the accounts are already in global memory) ----------------------------------------
  for (int a = lane; a < A; a += 32) {
    P.ord[aoff + a] = sm.ord[a];
    const uint32_t o = sm.ord[a];
    const bool last_one = w_qty(o) != 0u && sm.tail[(int)w_sell(o) * L + (int)w_tick(o)] == a;
    P.nxt[aoff + a] = last_one ? -1 : sm.nxt[a];
  }
  if (lane == 0) {
    int32_t* mo = P.mi32 + (size_t)m * MI32_STRIDE;
    mo[MI_LAST] = last;
#pragma unroll
    for (int j = 0; j < KS_HISTORY; ++j) mo[MI_HIST + j] = hist[j];
    mo[MI_TRADES] = fills;
    mo[MI_LASTV] = lastv;
    int64_t* m64 = P.mi64 + (size_t)m * MI64_STRIDE;
    m64[MI_SUMP] = value;
    m64[MI_SUMV] = sumv;
    m64[MI_HASH] = (int64_t)hash;
  }
  __syncwarp();
}

// Persistent: warp w of CTA b runs markets b * WPB + w, + grid * WPB, ...
__global__ void __launch_bounds__(1024) cda_kernel(CdaParams P, uint32_t n_steps, uint32_t stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int wpb = (int)blockDim.x >> 5;
  const CdaSmem sm = cda_carve(smem_raw + (size_t)warp * stride, P.A, P.L);
  const uint32_t s0 = (uint32_t)(*P.step);
  for (uint32_t m = blockIdx.x * wpb + warp; m < P.M; m += gridDim.x * wpb) cda_market(P, m, s0, n_steps, sm, lane);
}

__global__ void cda_bump_kernel(uint64_t* step, uint32_t n) { *step += n; }

}  // namespace
}  // namespace ks

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
struct ks_cda_ensemble {
  ks::CdaParams p;
  ks_cda_config cfg;
  unsigned char* ws;
  size_t bytes;
  int device, num_sms, wpb, grid;
  uint32_t stride;
  size_t smem;
};

namespace ks {
namespace {

struct CdaLayout {
  size_t ord, inv, cash, nxt, mi32, mi64, trace, ctrl, total;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

CdaLayout cda_layout(const ks_cda_config* c) {
  const size_t N = (size_t)c->n_markets * (size_t)c->A, M = c->n_markets;
  CdaLayout l;
  size_t o = 0;
  l.ord = o; o = al256(o + 4 * N);
  l.inv = o; o = al256(o + 4 * N);
  l.cash = o; o = al256(o + 8 * N);
  l.nxt = o; o = al256(o + 4 * N);
  l.mi32 = o; o = al256(o + 4 * M * MI32_STRIDE);
  l.mi64 = o; o = al256(o + 8 * M * MI64_STRIDE);
  l.trace = o; o = al256(o + 8 * (size_t)c->trace_markets * c->trace_steps);
  l.ctrl = o; o = al256(o + 64);  // err (u32) at +0, step (u64) at +8
  l.total = o;
  return l;
}

ks_status cfail(ks_status s, const char* msg) {
  internal_set_error(msg);
  return s;
}

ks_status ccuda(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  internal_set_error(buf);
  return KS_ERR_CUDA;
}

#define KSC_CUDA(call)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return ccuda(e_, #call);    \
  } while (0)

ks_status cda_validate(const ks_cda_config* c) {
  if (!c) return cfail(KS_ERR_INVALID_ARG, "config is NULL");
  if (c->n_markets == 0) return cfail(KS_ERR_INVALID_ARG, "n_markets must be >= 1");
  if (c->n_markets > (1u << 26)) return cfail(KS_ERR_UNSUPPORTED, "n_markets above 2^26");
  if ((uint64_t)c->market_base + c->n_markets > 0xFFFFFFFFull)
    return cfail(KS_ERR_INVALID_ARG, "market_base + n_markets above 2^32");
  if (c->L < 2 || c->L > KS_MAX_TICKS) return cfail(KS_ERR_UNSUPPORTED, "L outside [2, KS_MAX_TICKS]");
  if (c->A < 0 || c->A > KS_CDA_MAX_AGENTS) return cfail(KS_ERR_UNSUPPORTED, "A outside [0, KS_CDA_MAX_AGENTS]");
  if (c->mix_pct[0] + c->mix_pct[1] + c->mix_pct[2] != 100u)
    return cfail(KS_ERR_INVALID_ARG, "mix_pct must sum to 100");
  if (c->zi_offset < 0 || c->zi_offset > KS_MAX_TICKS || c->mom_offset_max < 0 || c->mom_offset_max > KS_MAX_TICKS ||
      c->mr_offset_max < 0 || c->mr_offset_max > KS_MAX_TICKS)
    return cfail(KS_ERR_INVALID_ARG, "offset out of range");
  if (c->zi_qmax < 1 || c->rb_qmax < 1) return cfail(KS_ERR_INVALID_ARG, "qmax must be >= 1");
  if (c->zi_qmax > KS_MAX_QTY || c->rb_qmax > KS_MAX_QTY) return cfail(KS_ERR_UNSUPPORTED, "qmax above 255");
  if (c->mom_lookback < 1 || c->mom_lookback > KS_HISTORY - 1)
    return cfail(KS_ERR_INVALID_ARG, "mom_lookback must be in [1, 8]");
  if (c->trace_markets > c->n_markets) return cfail(KS_ERR_INVALID_ARG, "trace_markets above n_markets");
  if (c->trace_markets != 0 && c->trace_steps == 0) return cfail(KS_ERR_INVALID_ARG, "trace_steps must be > 0 when tracing");
  // one step's volume is at most A orders of at most 255
  if ((int64_t)c->A * KS_MAX_QTY >= (1ll << 31)) return cfail(KS_ERR_UNSUPPORTED, "A * 255 above 2^31");
  return KS_OK;
}

}  // namespace
}  // namespace ks

extern "C" {

ks_status ks_cda_workspace_size(const ks_cda_config* cfg, size_t* bytes) {
  using namespace ks;
  if (!bytes) return cfail(KS_ERR_INVALID_ARG, "bytes is NULL");
  const ks_status s = cda_validate(cfg);
  if (s != KS_OK) return s;
  *bytes = cda_layout(cfg).total;
  return KS_OK;
}

ks_status ks_cda_create(const ks_cda_config* cfg, void* dev_workspace, size_t ws_bytes, void* cuda_stream,
                        ks_cda_ensemble** out) {
  using namespace ks;
  if (!out || !dev_workspace) return cfail(KS_ERR_INVALID_ARG, "NULL argument");
  ks_status s = cda_validate(cfg);
  if (s != KS_OK) return s;
  const CdaLayout lay = cda_layout(cfg);
  if (ws_bytes < lay.total) return cfail(KS_ERR_WORKSPACE_TOO_SMALL, "workspace smaller than ks_cda_workspace_size");
  if (((uintptr_t)dev_workspace & 255u) != 0) return cfail(KS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  ks_cda_ensemble* e = new (std::nothrow) ks_cda_ensemble();
  if (!e) return cfail(KS_ERR_INVALID_ARG, "out of host memory");
  e->cfg = *cfg;
  e->ws = (unsigned char*)dev_workspace;
  e->bytes = ws_bytes;
  int max_optin = 0;
  cudaError_t ce = cudaGetDevice(&e->device);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, e->device);
  if (ce != cudaSuccess) {
    delete e;
    return ccuda(ce, "device query");
  }
  int smem_sm = 0;
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, e->device);
  if (ce != cudaSuccess) {
    delete e;
    return ccuda(ce, "device query");
  }
  size_t o[7];
  const size_t per = cda_smem_layout(cfg->A, cfg->L, o);
  e->stride = (uint32_t)per;
  // One CTA per SM holds as many books (warps) as the shared memory fits, up to
  // 32; of those, as few as keep the number of rounds over the markets.
  const size_t room = std::min<size_t>((size_t)max_optin, smem_sm > 1024 ? (size_t)smem_sm - 1024 : 0);
  const int fit = (int)std::min<size_t>(32, room / per);
  if (fit < 1) {
    delete e;
    return cfail(KS_ERR_UNSUPPORTED, "one market's book does not fit the shared memory of a CTA");
  }
  const int64_t per_round = (int64_t)fit * e->num_sms;
  const int64_t rounds = ((int64_t)cfg->n_markets + per_round - 1) / per_round;
  const int64_t need = ((int64_t)cfg->n_markets + rounds * e->num_sms - 1) / (rounds * e->num_sms);
  e->wpb = (int)std::max<int64_t>(1, std::min<int64_t>(fit, need));
  e->smem = (size_t)e->wpb * per;
  ce = cudaFuncSetAttribute(cda_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem);
  int occ = 0;
  if (ce == cudaSuccess) ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cda_kernel, 32 * e->wpb, e->smem);
  if (ce != cudaSuccess || occ < 1) {
    delete e;
    return ce != cudaSuccess ? ccuda(ce, "cda occupancy") : cfail(KS_ERR_UNSUPPORTED, "CDA launch does not fit an SM");
  }
  const int64_t ctas = ((int64_t)cfg->n_markets + e->wpb - 1) / e->wpb;
  e->grid = (int)std::min<int64_t>(ctas, (int64_t)occ * e->num_sms);

  CdaParams& p = e->p;
  memset(&p, 0, sizeof(p));
  p.M = cfg->n_markets;
  p.market_base = cfg->market_base;
  p.L = cfg->L;
  p.A = cfg->A;
  const uint32_t key0 = (uint32_t)(cfg->seed & 0xffffffffu), key1 = (uint32_t)(cfg->seed >> 32);
  for (int r = 0; r < 10; ++r) {
    p.rk[2 * r] = key0 + (uint32_t)r * PH_WA;
    p.rk[2 * r + 1] = key1 + (uint32_t)r * PH_WB;
  }
  p.cancel_thr = cfg->cancel_thresh_q32;
  p.rc.zi_off = cfg->zi_offset;
  p.rc.zi_n = 2u * (uint32_t)cfg->zi_offset + 1u;
  p.rc.zi_qmax = (uint32_t)cfg->zi_qmax;
  p.rc.mom_n = (uint32_t)cfg->mom_offset_max + 1u;
  p.rc.mr_n = (uint32_t)cfg->mr_offset_max + 1u;
  p.rc.rb_qmax = (uint32_t)cfg->rb_qmax;
  p.mom_lb = cfg->mom_lookback;
  p.trace_markets = cfg->trace_markets;
  p.trace_steps = cfg->trace_steps;
  unsigned char* w = e->ws;
  p.ord = (uint32_t*)(w + lay.ord);
  p.inv = (int32_t*)(w + lay.inv);
  p.cash = (int64_t*)(w + lay.cash);
  p.nxt = (int32_t*)(w + lay.nxt);
  p.mi32 = (int32_t*)(w + lay.mi32);
  p.mi64 = (int64_t*)(w + lay.mi64);
  p.trace = (int32_t*)(w + lay.trace);
  p.err = (uint32_t*)(w + lay.ctrl);
  p.step = (const uint64_t*)(w + lay.ctrl + 8);

  // the initial state of the main model: classes, fundamentals, opening tick, no orders
  DevParams d;
  memset(&d, 0, sizeof(d));
  d.M = p.M;
  d.market_base = p.market_base;
  d.L_all = p.L;
  d.A_all = p.A;
  d.key0 = key0;
  d.key1 = key1;
  d.mix0 = cfg->mix_pct[0];
  d.mix01 = cfg->mix_pct[0] + cfg->mix_pct[1];
  d.mlp_pct = 0;
  d.slot = p.ord;
  d.inv = p.inv;
  d.cash = p.cash;
  d.mi32 = p.mi32;
  d.mi64 = p.mi64;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  ce = cudaMemsetAsync(w + lay.ctrl, 0, 64, st);
  if (ce == cudaSuccess && lay.ctrl > lay.trace) ce = cudaMemsetAsync(w + lay.trace, 0, lay.ctrl - lay.trace, st);
  if (ce == cudaSuccess && lay.mi32 > lay.nxt) ce = cudaMemsetAsync(w + lay.nxt, 0xFF, lay.mi32 - lay.nxt, st);
  if (ce == cudaSuccess)
    ce = internal_init_state(d, (int)std::min<uint32_t>(p.M, 8u * (uint32_t)e->num_sms), st);
  if (ce != cudaSuccess) {
    delete e;
    return ccuda(ce, "CDA initial state");
  }
  *out = e;
  return KS_OK;
}

ks_status ks_cda_step_n(ks_cda_ensemble* e, uint32_t n_steps, void* cuda_stream) {
  using namespace ks;
  if (!e) return cfail(KS_ERR_INVALID_ARG, "ensemble is NULL");
  if (n_steps == 0) return KS_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cda_kernel<<<e->grid, 32 * e->wpb, e->smem, st>>>(e->p, n_steps, e->stride);
  KSC_CUDA(cudaGetLastError());
  cda_bump_kernel<<<1, 1, 0, st>>>((uint64_t*)e->p.step, n_steps);
  KSC_CUDA(cudaGetLastError());
  return KS_OK;
}

ks_status ks_cda_read_state(ks_cda_ensemble* e, const ks_cda_state_view* v, void* cuda_stream) {
  using namespace ks;
  if (!e || !v) return cfail(KS_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t N = (size_t)e->p.M * (size_t)e->p.A, M = e->p.M;
  if (v->order && N) KSC_CUDA(cudaMemcpyAsync(v->order, e->p.ord, 4 * N, cudaMemcpyDeviceToHost, st));
  if (v->inventory && N) KSC_CUDA(cudaMemcpyAsync(v->inventory, e->p.inv, 4 * N, cudaMemcpyDeviceToHost, st));
  if (v->cash && N) KSC_CUDA(cudaMemcpyAsync(v->cash, e->p.cash, 8 * N, cudaMemcpyDeviceToHost, st));
  if (v->next && N) KSC_CUDA(cudaMemcpyAsync(v->next, e->p.nxt, 4 * N, cudaMemcpyDeviceToHost, st));
  struct F32 { int32_t* dst; int col; int width; };
  const F32 f32[] = {{v->last_tick, MI_LAST, 1}, {v->history, MI_HIST, KS_HISTORY}, {v->fundamental, MI_FUND, 1},
                     {v->fills, MI_TRADES, 1}, {v->last_volume, MI_LASTV, 1}};
  for (const F32& f : f32)
    if (f.dst)
      KSC_CUDA(cudaMemcpy2DAsync(f.dst, 4 * f.width, e->p.mi32 + f.col, 4 * MI32_STRIDE, 4 * f.width, M,
                                 cudaMemcpyDeviceToHost, st));
  struct F64 { void* dst; int col; };
  const F64 f64[] = {{v->traded_value, MI_SUMP}, {v->sum_volume, MI_SUMV}, {v->trace_hash, MI_HASH}};
  for (const F64& f : f64)
    if (f.dst)
      KSC_CUDA(cudaMemcpy2DAsync(f.dst, 8, e->p.mi64 + f.col, 8 * MI64_STRIDE, 8, M, cudaMemcpyDeviceToHost, st));
  if (v->step) KSC_CUDA(cudaMemcpyAsync(v->step, e->p.step, 8, cudaMemcpyDeviceToHost, st));
  const size_t tb = 8 * (size_t)e->p.trace_markets * e->p.trace_steps;
  if (v->trace && tb) KSC_CUDA(cudaMemcpyAsync(v->trace, e->p.trace, tb, cudaMemcpyDeviceToHost, st));
  KSC_CUDA(cudaStreamSynchronize(st));
  return KS_OK;
}

ks_status ks_cda_sync(ks_cda_ensemble* e, void* cuda_stream, uint32_t timeout_ms) {
  using namespace ks;
  if (!e) return cfail(KS_ERR_INVALID_ARG, "ensemble is NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t ev;
  KSC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t ce = cudaEventRecord(ev, st);
  if (ce != cudaSuccess) {
    cudaEventDestroy(ev);
    return ccuda(ce, "cudaEventRecord");
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    ce = cudaEventQuery(ev);
    if (ce == cudaSuccess) break;
    if (ce != cudaErrorNotReady) {
      cudaEventDestroy(ev);
      return ccuda(ce, "cudaEventQuery");
    }
    if (timeout_ms) {
      const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
      if (ms.count() >= (long long)timeout_ms) {
        cudaEventDestroy(ev);
        return cfail(KS_ERR_TIMEOUT, "ks_cda_sync deadline passed before the stream finished");
      }
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  uint32_t word = 0;
  KSC_CUDA(cudaMemcpyAsync(&word, e->p.err, 4, cudaMemcpyDeviceToHost, st));
  KSC_CUDA(cudaStreamSynchronize(st));
  if (word) {
    char buf[64];
    snprintf(buf, sizeof(buf), "device error word 0x%x", word);
    internal_set_error(buf);
    return KS_ERR_DEVICE_FAULT;
  }
  return KS_OK;
}

ks_status ks_cda_destroy(ks_cda_ensemble* e) {
  delete e;
  return KS_OK;
}

}  // extern "C"
