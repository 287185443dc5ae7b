// ks_market.cuh -- one market's persistent call-auction loop (sm_103a).
//
// A group of GT threads (a whole CTA, or a slice of one when several small
// markets share a CTA) owns one market at a time and keeps it on chip for all
// n steps of a call (the paper's Algorithm 1 and Sec. III-B residency,
// re-shaped for GB300): thread t owns agents [t*AK, t*AK+AK) and ticks
// [t*LT, t*LT+LT) of the aggregated book in shared memory.  An agent's order
// word lives in a register of its thread; its inventory and cash either in
// registers too (inventory, and the cash of the current 1024-step window
// over a 64-bit total in a thread-private shared-memory column) or, where
// the CTA's register budget is smaller, in thread-private shared-memory
// columns (accounts_in_registers).
//
// Step s, between four group barriers:
//   B1  all orders of step s are in the book (shared atomics)      (Alg. 1, Phase 3)
//   B2  per-thread tick sums, warp shuffle scans; warp totals published
//   B3  D_cum / S_cum / V = min per tick (Eq. 1-2); warp redux.sync of the
//       best V and its lowest / highest tick; one 64-bit shared atomicMax per
//       warp for each.  The lowest maximiser of V is p* (ties to the lowest
//       tick, Sec. III-D) and the marginal sell tick; the highest maximiser is
//       the marginal buy tick.                                    (Phase 4)
//   B5  tick owners update the resting book without atomics and publish the
//       rationed remainders at the marginal ticks; each thread sums its
//       orders resting at the marginal ticks for one ordered block scan.
//   then one pass per agent fills step s (price priority, then ascending
//   agent index at the marginal ticks, Sec. IV-C) and draws step s+1's
//   cancellation and new order (Philox4x32-10).                  (Phase 5)
// Global memory is touched only when a market is loaded and stored, so the
// traffic does not grow with the number of steps (Sec. III-F).
#pragma once

#include <stdint.h>

#include "ks_device.cuh"
#include "ks_mlp.cuh"

namespace ks {

// Cash moves into 32-bit per-agent registers between flushes into the 64-bit
// total: one step changes an agent's cash by at most 4095 * 255 < 2^20 tick
// units, so 1024 steps stay below 2^31.
constexpr uint32_t CASH_FLUSH_STEPS = 1024;

// Registers a thread may use when min_ctas CTAs of cta_threads threads share
// an SM's 65536 (the launch bounds), at most 255.
__host__ __device__ constexpr int thread_reg_budget(int cta_threads, int min_ctas) {
  return 65536 / (cta_threads * min_ctas) < 255 ? 65536 / (cta_threads * min_ctas) : 255;
}

// Where the agents' inventory and cash live: registers when order word,
// inventory and pending cash (3 per agent) and about 56 more fit the budget,
// shared memory otherwise.  Policy kernels keep them in shared memory, where
// the policy rows read the inventory.
__host__ __device__ constexpr bool accounts_in_registers(int reg_budget, int ak, bool mlp) {
  return !mlp && 3 * ak + 56 <= reg_budget;
}

struct Smem {
  int64_t* cash;          // [AK][NT] thread-private columns: cash (registers accounts: up to the last flush)
  unsigned long long* kx; // [2 parities][4]: lowest / highest maximiser keys, tie key
  int32_t* inv;           // [AK][NT] thread-private columns of inventory (shared-memory accounts)
  int32_t* book;          // BUY[p] at 2p, SELL[p] at 2p + 1, p < book_len(Lmax)
  int32_t* wD;            // [32] warp totals of BUY
  int32_t* wS;            // [32] warp totals of SELL
  uint32_t* wMB;          // [32] warp totals of marginal buy quantity
  uint32_t* wMS;          // [32] warp totals of marginal sell quantity
  int32_t* rem;           // [2]: R_b, R_s (units filled at the marginal buy / sell tick)
  int32_t* rng;           // [2 parities][2]: lowest / highest tick holding a resting order after a step
  int32_t* feat;          // [8]: resting sell qty at last+1..+4, buy qty at last-1..-4 (policy inputs)
  int32_t* wR;            // [32] warp totals of policy rows
  uint4* drow;            // [8] decision rows per (agent class, side coin) for the next orders
  uint32_t* dsell;        // [8] their side bits
  float* cvec;            // [64] layer-1 pre-activation shared by the market's agents (policy kernels)
  uint32_t* rowbuf;       // [NT * AK] policy rows: agent index, then the decision (policy kernels)
};

// Shared memory of one market group; `mlp` adds the policy buffers,
// `inv_col` the inventory columns (shared-memory accounts).
__host__ __device__ inline size_t market_smem_layout(int nt, int ak, int Lmax, bool mlp, bool inv_col, size_t* o) {
  size_t off = 0;
  o[0] = off; off += (size_t)8 * ak * nt;                // cash
  o[1] = off; off += (size_t)8 * 8;                      // kx
  o[2] = off; off += inv_col ? (size_t)4 * ak * nt : 0;  // inv
  o[3] = off; off += (size_t)4 * 2 * book_len(Lmax);     // book
  o[4] = off; off += (size_t)4 * 32 * 4 + 4 * 8;         // wD, wS, wMB, wMS, rem, rng
  o[5] = off; off += (size_t)4 * 8 + 4 * 32 + 8 * 16 + 8 * 4;  // feat, wR, drow, dsell
  o[6] = off; off += mlp ? (size_t)4 * 64 : 0;           // cvec
  o[7] = off; off += mlp ? (size_t)4 * ak * nt : 0;      // rowbuf
  return (off + 15) & ~(size_t)15;
}

// Shared memory of one market group of gt threads under a register budget.
__host__ __device__ inline size_t group_smem_layout(int reg_budget, int gt, int ak, int Lmax, bool mlp, size_t* o) {
  return market_smem_layout(gt, ak, Lmax, mlp, !accounts_in_registers(reg_budget, ak, mlp), o);
}

template <int NT, int AK, bool MLP, bool INV_COL>
__device__ __forceinline__ Smem carve(unsigned char* raw, int Lmax) {
  size_t o[8];
  market_smem_layout(NT, AK, Lmax, MLP, INV_COL, o);
  Smem s;
  s.cash = reinterpret_cast<int64_t*>(raw + o[0]);
  s.kx = reinterpret_cast<unsigned long long*>(raw + o[1]);
  s.inv = reinterpret_cast<int32_t*>(raw + o[2]);
  s.book = reinterpret_cast<int32_t*>(raw + o[3]);
  s.wD = reinterpret_cast<int32_t*>(raw + o[4]);
  s.wS = s.wD + 32;
  s.wMB = reinterpret_cast<uint32_t*>(s.wD + 64);
  s.wMS = s.wMB + 32;
  s.rem = s.wD + 128;
  s.rng = s.wD + 132;
  s.feat = reinterpret_cast<int32_t*>(raw + o[5]);
  s.wR = s.feat + 8;
  s.drow = reinterpret_cast<uint4*>(s.wR + 32);
  s.dsell = reinterpret_cast<uint32_t*>(s.drow + 8);
  s.cvec = reinterpret_cast<float*>(raw + o[6]);
  s.rowbuf = reinterpret_cast<uint32_t*>(raw + o[7]);
  return s;
}

// Barrier of the GT threads owning a market: a warp-sized group uses
// __syncwarp, larger groups a named barrier (id 0 only when the group is the
// whole CTA).
template <int GT>
__device__ __forceinline__ void gsync(int bar) {
  if constexpr (GT == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(GT) : "memory");
  }
}

// Add the order word's quantity at its (side, tick).  With AGGR, lanes of the
// warp holding the same (side, tick) first combine their quantities
// (__match_any_sync + __reduce_add_sync) and one lane issues the atomic.
template <bool AGGR>
__device__ __forceinline__ void book_add(uint32_t book_s, bool valid, uint32_t w) {
  const uint32_t i = w_bidx(w);
  const int q = (int)w_qty(w);
  if constexpr (AGGR) {
    const uint32_t key = valid ? i : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int tot = (int)__reduce_add_sync(peers, (unsigned)q);
    const int leader = __ffs(peers) - 1;
    red_add_if(book_s + 4u * i, tot, valid && (int)(threadIdx.x & 31) == leader);
  } else {
    red_add_if(book_s + 4u * i, q, valid);
  }
}

// Uniform per-step inputs of the agent rules.
struct StepRules {
  StepKey sk;
  int last;
  int side_mom;  // 0 buy, 1 sell, -1 undecided
  int side_mr;
};

// Market-level policy inputs of a step: clearing-tick returns, last volume
// (registers) and resting depth around the last tick (shared memory).
struct StepFeat {
  int h[8];
  int lastv;
  const int32_t* depth;
};

// Appends one rule-decision record (the behaviour-cloning data).
__device__ __forceinline__ void record_decision(const DevParams& P, const StepFeat& f, int inv, uint32_t w, int last) {
  const unsigned long long i = atomicAdd(P.rec_count, 1ull);
  if (i >= P.rec_cap) return;
  int32_t* r = P.rec + i * KS_RECORD_WORDS;
#pragma unroll
  for (int j = 0; j < 8; ++j) r[j] = f.h[j];
  r[8] = inv;
  r[9] = f.lastv;
#pragma unroll
  for (int j = 0; j < 8; ++j) r[10 + j] = f.depth[j];
  r[18] = (int)w_sell(w);
  const int toward = w_sell(w) ? last - (int)w_tick(w) : (int)w_tick(w) - last;  // toward the opposite side
  r[19] = min(max(toward, -MLP_OFF_MAX), MLP_OFF_MAX) + MLP_OFF_MAX;
  r[20] = (int)w_qty(w);
  r[21] = (int)w_class(w);
}

// Step-s order of one agent: cancellation of its working order (carried
// books; cthr = 0 never cancels), then a new order if it has none.  x0 is the
// agent's first Philox word (StepKey::c0 ^ agent).  Returns the new order
// word.  With MLP, a policy-driven agent without an order sets `policy`
// instead of deciding, and rule decisions of recorded agents are appended.
template <bool AGGR, bool MLP = false, int CM = 2>
__device__ __forceinline__ uint32_t order_agent(uint32_t sl, int a, uint32_t x0, bool valid, const StepRules& sr,
                                                uint32_t cthr, int L, const uint4* drow, const uint32_t* dsell,
                                                uint32_t book_s,
                                                const uint32_t* rk, bool* policy = nullptr,
                                                const DevParams* P = nullptr, const StepFeat* f = nullptr,
                                                int inv = 0) {
  const uint4 w = step_draw_x0(sr.sk, x0, rk);
  const uint32_t q = w_qty(sl);
  const bool cancel = q != 0u && w.x < cthr;
  red_add_if(book_s + 4u * w_bidx(sl), -(int)q, cancel);
  const bool empty = valid && (q == 0u || cancel);
  // without a policy network the policy flag is ignored: every empty agent
  // decides by its rule (no flag test: 1.9% on the 8192-market workload)
  const bool dec = MLP ? (empty && !(sl & W_MLP)) : empty;
  const uint32_t ns = decide_rows(sl, w, drow, dsell, L);
  book_add<AGGR>(book_s, dec, ns);
  if constexpr (MLP) {
    *policy = empty && (sl & W_MLP);
    if (dec && (uint32_t)a < P->rec_agents) record_decision(*P, *f, inv, ns, sr.last);
  }
  // carried-book rule kernels: an agent outside the market holds a zero word
  // (no cancellation), and a cancelled agent decides, so an agent that does not
  // decide keeps its word (0.4%)
  if constexpr (!MLP && CM != 2) return dec ? ns : sl;
  return dec ? ns : (cancel ? (sl & W_STATIC) : sl);
}

__device__ __forceinline__ StepRules step_rules(const DevParams& P, uint32_t s, uint32_t gm, int h0, int hlb, int last,
                                                int fund) {
  StepRules r;
  r.sk = step_key(s, gm, 0u, P.rk);
  const int ret = h0 - hlb;
  r.side_mom = ret > 0 ? 0 : (ret < 0 ? 1 : -1);
  r.side_mr = last < fund ? 0 : (last > fund ? 1 : -1);
  r.last = last;
  return r;
}

// hist[lookback] with a compile-time index per candidate, so the history
// stays in registers.
__device__ __forceinline__ int hist_at(const int (&hist)[KS_HISTORY], int lb) {
  int h = hist[1];
#pragma unroll
  for (int i = 2; i < KS_HISTORY; ++i) h = (lb == i) ? hist[i] : h;
  return h;
}


// Policy decisions of one step for the agents flagged in `pflags` (bit k =
// agent a0 + k): rows are compacted in agent order, the group's warpgroups
// evaluate them in tiles of 128 (tile i on warpgroup i mod mw.nwg, each
// with its own activation buffer, accumulator columns and mbarrier in `mw`)
// on the tensor cores and sample the actions (Philox stream 3 of step
// sdec), then the owners place the orders.
// The inventories of the flagged agents are in sm.inv; thread t owns agents
// [t * akeff, t * akeff + akeff).
template <int NT, int AK>
__device__ __forceinline__ void policy_phase(const DevParams& P, const Smem& sm, MlpWG& mw, const unsigned char* sw,
                                             uint32_t (&slot)[AK], uint32_t pflags, int t, int bar, int a0, int A,
                                             int L, uint32_t sdec, uint32_t gm, const StepFeat& f, int last,
                                             int64_t aoff, bool traced, int32_t* book, int akeff) {
  constexpr int NW = NT / 32;
  const int lane = t & 31;
  const int wid = t >> 5;
  const int cnt = __popc(pflags);
  int inc = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) sm.wR[wid] = inc;
  if (t < MLP_H) {
    // layer-1 pre-activation of everything but the inventory input
    const float* w1 = reinterpret_cast<const float*>(sw + MLP_SM_W1) + t * MLP_IN;
    const float* b1 = reinterpret_cast<const float*>(sw + MLP_SM_B);
    const float inv8A = 1.0f / (8.0f * (float)max(A, 1));
    const float inv4A = 1.0f / (4.0f * (float)max(A, 1));
    float c = b1[t];
#pragma unroll
    for (int j = 0; j < 8; ++j) c = fmaf(w1[j], (float)f.h[j] * 0.125f, c);
    c = fmaf(w1[9], (float)f.lastv * inv8A, c);
#pragma unroll
    for (int j = 0; j < 8; ++j) c = fmaf(w1[10 + j], (float)f.depth[j] * inv4A, c);
    sm.cvec[t] = c;
  }
  gsync<NT>(bar);
  const int before = inc - cnt + (int)__reduce_add_sync(0xffffffffu, lane < wid ? (unsigned)sm.wR[lane] : 0u);
  const int total = (int)__reduce_add_sync(0xffffffffu, lane < NW ? (unsigned)sm.wR[lane] : 0u);
  int r = before;
#pragma unroll
  for (int k = 0; k < AK; ++k)
    if ((pflags >> k) & 1u) sm.rowbuf[r++] = (uint32_t)(a0 + k);
  gsync<NT>(bar);
  if (t == 0 && total > 0 && P.pol_count) atomicAdd(P.pol_count, (unsigned long long)total);
  if (total > 0 && mw.wg < mw.nwg) {
    // stream-3 draws (counter (sdec, agent, market, 3)): the agent-independent
    // parts of rounds 1-3 once per step, as for the per-step draws
    const StepKey sk3 = step_key(sdec, gm, 3u, P.rk);
    for (int tile = mw.wg; tile * 128 < total; tile += mw.nwg) {
      const int row = tile * 128 + (t & 127);
      const bool valid = row < total;
      const int a = valid ? (int)sm.rowbuf[row] : 0;
      const int ta = a / akeff;
      const int inv = valid ? sm.inv[(a - ta * akeff) * NT + ta] : 0;
      float z[MLP_OUT];
      mlp_tile_logits(mw, sw, sm.cvec, (float)inv * (1.0f / 256.0f), z, P.err);
      if (valid) {
        const uint4 w = step_draw_x0(sk3, sk3.c0 ^ (uint32_t)a, P.rk);
        sm.rowbuf[row] = mlp_decision(z, w, last, L, P.rb_qmax);
        if (traced && P.logit_trace && sdec < P.trace_steps) {
          float* zo = P.logit_trace + ((size_t)sdec * P.dec_trace_agents + (size_t)(aoff + a)) * MLP_OUT;
#pragma unroll
          for (int i = 0; i < MLP_OUT; ++i) zo[i] = z[i];
        }
      }
    }
  }
  gsync<NT>(bar);
  r = before;
#pragma unroll
  for (int k = 0; k < AK; ++k) {
    if ((pflags >> k) & 1u) {
      const uint32_t d = sm.rowbuf[r++];
      if (!(d & KS_DECISION_PASS)) {
        slot[k] = (slot[k] & W_STATIC) | d;
        atomicAdd(book + w_bidx(d), (int)w_qty(d));
      }
      if (traced && P.dec_trace && sdec < P.trace_steps)
        P.dec_trace[(size_t)sdec * P.dec_trace_agents + (size_t)(aoff + a0 + k)] = d;
    }
  }
}

// Resting depth around tick nl from the book (the policy inputs): each entry
// has exactly one writer, the owner of its tick or thread 0 off the grid.
__device__ __forceinline__ void publish_depth(const Smem& sm, const int32_t* book, int L, int nl, int p0, int LT,
                                              int t) {
  for (int i = 0; i < LT; ++i) {
    const int p = p0 + i;
    if (p < L) {
      if (p > nl && p <= nl + 4) sm.feat[p - nl - 1] = book[bidx(1, p)];
      if (p < nl && p >= nl - 4) sm.feat[4 + nl - p - 1] = book[bidx(0, p)];
    }
  }
  if (t == 0) {
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
      if (nl + k >= L) sm.feat[k - 1] = 0;
      if (nl - k < 0) sm.feat[4 + k - 1] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// One clearing of the book (Eq. 1-2, Phase 4) and the residual update
// (Phase 5).  The thread owns ticks [p0, p0 + LT).  LTC > 0: LT == LTC and
// the (BUY, SELL) pairs are loaded once with vector accesses and kept in
// registers; LTC == 0: any LT, scalar accesses.
// ---------------------------------------------------------------------------
struct ClearOut {
  int vstar, p_lo, p_hi, pstar;
};

// (BUY, SELL) pairs of N consecutive ticks starting at word src (8N bytes, aligned to min(16, 8N)).
template <int N>
__device__ __forceinline__ void ld_pairs(const int32_t* src, int* b, int* s) {
  if constexpr (N == 1) {
    const int2 a = *reinterpret_cast<const int2*>(src);
    b[0] = a.x; s[0] = a.y;
  } else {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const int4 a = *reinterpret_cast<const int4*>(src + 2 * i);
      b[i] = a.x; s[i] = a.y; b[i + 1] = a.z; s[i + 1] = a.w;
    }
  }
}

template <int N>
__device__ __forceinline__ void st_pairs(int32_t* dst, const int* b, const int* s) {
  if constexpr (N == 1) {
    *reinterpret_cast<int2*>(dst) = make_int2(b[0], s[0]);
  } else {
#pragma unroll
    for (int i = 0; i < N; i += 2) *reinterpret_cast<int4*>(dst + 2 * i) = make_int4(b[i], s[i], b[i + 1], s[i + 1]);
  }
}

// The group clears the tick region [plo, pend): the whole grid (plo = 0,
// pend = L) or a window that holds every order of the step (all ticks
// outside it are empty, so D_cum and S_cum there are constant, V = 0, and
// nothing changes).  Ticks in [L, pend) lie in the zeroed padding of the
// book.  The lowest and highest ticks still holding an order after the
// residual update go to rng_next (shared-memory atomicMin / atomicMax).
template <int NT, int LTC, bool FEAT>
__device__ __forceinline__ ClearOut clear_step(const Smem& sm, int32_t* book, int L, int LT, int p0, int plo,
                                               int pend, int t, int bar, unsigned long long* kx,
                                               unsigned long long* kx_next, int32_t* rng_next, bool tie1, bool carry,
                                               int last) {
  const int lane = t & 31;
  const int wid = t >> 5;
  constexpr int R = LTC > 0 ? LTC : 1;
  int bv[R], sv[R];
  const bool mine = p0 < pend;  // vector path: all LTC ticks of an owning thread lie in the region
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
    for (int i = 0; i < LT; ++i) {
      const int p = p0 + i;
      if (p < pend) {
        sumB += book[2 * p];
        sumS += book[2 * p + 1];
      }
    }
  }
  int sufB = sumB, preS = sumS;  // inclusive warp suffix (BUY) / prefix (SELL) scans
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int vb = __shfl_down_sync(0xffffffffu, sufB, d);
    const int vs = __shfl_up_sync(0xffffffffu, preS, d);
    if (lane + d < 32) sufB += vb;
    if (lane >= d) preS += vs;
  }
  if (lane == 0) sm.wD[wid] = sufB;
  if (lane == 31) sm.wS[wid] = preS;
  gsync<NT>(bar);  // B2
  const int offD = (int)__reduce_add_sync(0xffffffffu, (lane < NT / 32 && lane > wid) ? (unsigned)sm.wD[lane] : 0u);
  const int offS = (int)__reduce_add_sync(0xffffffffu, (lane < wid) ? (unsigned)sm.wS[lane] : 0u);
  const int D0 = offD + sufB;          // D_cum at my first tick
  const int Sb0 = offS + preS - sumS;  // S_cum just below my first tick
  // A tick range with no orders: D and S are constant on it, so V is
  // min(D0, Sb0) on every tick, its lowest and highest maximisers are the
  // range's ends, and nothing in it changes (policy depth there is zero).
  const int cnt = LTC > 0 ? (mine ? LTC : 0) : max(0, min(LT, pend - p0));  // ticks in the region
  const bool idle = cnt > 0 && sumB == 0 && sumS == 0;
  {
    int D = D0, Sb = Sb0;
    int bestV = -1, lo = 4095, hi = 0;
    unsigned long long kT = 0ull;
    const int n = idle ? 0 : (LTC > 0 ? (mine ? LTC : 0) : LT);
    if (idle) {
      bestV = min(D0, Sb0);
      lo = p0;
      hi = p0 + cnt - 1;
      if (tie1) {
        const int imb = min(abs(D0 - Sb0), (1 << 22) - 1);
        kT = ((unsigned long long)(uint32_t)bestV << 34) | ((unsigned long long)((1 << 22) - 1 - imb) << 12) |
             (4095u - p0);
      }
    }
#pragma unroll
    for (int i = 0; i < (LTC > 0 ? LTC : 1); ++i) {
      // LTC == 0 runs this body in the loop below instead
      if (LTC > 0 && i < n) {
        const int p = p0 + i;
        const int S = Sb + sv[i];
        const int v = min(D, S);
        if (v > bestV) { bestV = v; lo = p; }
        if (v >= bestV) hi = p;
        if (tie1) {
          const int imb = min(abs(D - S), (1 << 22) - 1);
          const unsigned long long tk = ((unsigned long long)(uint32_t)v << 34) |
                                        ((unsigned long long)((1 << 22) - 1 - imb) << 12) | (4095u - p);
          kT = tk > kT ? tk : kT;
        }
        D -= bv[i];
        Sb = S;
      }
    }
    if constexpr (LTC == 0) {
      for (int i = 0; i < n; ++i) {
        const int p = p0 + i;
        if (p < pend) {
          const int b = book[2 * p];
          const int S = Sb + book[2 * p + 1];
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
        }
      }
    }
    const int vw = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(bestV, 0));
    const bool top = bestV == vw;
    const uint32_t low = __reduce_min_sync(0xffffffffu, top ? (unsigned)lo : 4095u);
    const uint32_t high = __reduce_max_sync(0xffffffffu, top ? (unsigned)hi : 0u);
    if (tie1) {
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, kT, d);
        kT = o > kT ? o : kT;
      }
    }
    if (lane == 0) {
      atomicMax(kx + 0, ((unsigned long long)(uint32_t)vw << 12) | (4095u - low));
      atomicMax(kx + 1, ((unsigned long long)(uint32_t)vw << 12) | high);
      if (tie1) atomicMax(kx + 2, kT);
    }
  }
  gsync<NT>(bar);  // B3
  ClearOut c;
  const unsigned long long kLo = kx[0], kHi = kx[1];
  c.vstar = (int)(kLo >> 12);
  c.p_lo = 4095 - (int)(kLo & 4095u);
  c.p_hi = (int)(kHi & 4095u);
  c.pstar = tie1 ? 4095 - (int)(kx[2] & 4095u) : c.p_lo;
  const bool trade = c.vstar > 0;
  if (t < 4) kx_next[t] = 0ull;  // reset the other parity for the next step

  // Residual book per tick, without atomics (Phase 5): the owners of the
  // marginal ticks publish R_b = V* - D_cum[p_hi + 1] and R_s = V* - S_cum[p_lo - 1];
  // a carried book keeps what did not trade, a discarded book is emptied.
  const int nl = trade ? c.pstar : last;  // last clearing tick after this step (policy depth)
  int rmin = 0x7FFFFFFF, rmax = -1;        // this thread's ticks still holding an order
  if (idle) {
    // nothing rests here.  A marginal tick holds orders (D_cum drops right after
    // p_hi, so BUY[p_hi] > 0; S_cum rises at p_lo, so SELL[p_lo] > 0), hence lies
    // in no empty range; the remainders below keep the rule explicit regardless.
    if (trade && c.p_hi >= p0 && c.p_hi < p0 + cnt) sm.rem[0] = c.vstar - D0;
    if (trade && c.p_lo >= p0 && c.p_lo < p0 + cnt) sm.rem[1] = c.vstar - Sb0;
    if constexpr (FEAT) {
      // the policy depth around the last tick: zero on an empty range
      const int f0 = max(p0, nl - 4), f1 = min(p0 + cnt - 1, nl + 4);
      for (int p = f0; p <= f1; ++p) {
        if (p > nl) sm.feat[p - nl - 1] = 0;
        if (p < nl) sm.feat[4 + nl - p - 1] = 0;
      }
    }
  } else if constexpr (LTC > 0) {
    if (mine) {
      int D = D0, Sb = Sb0;
#pragma unroll
      for (int i = 0; i < LTC; ++i) {
        const int p = p0 + i;
        const int b = bv[i], s = sv[i];
        int nb = b, ns = s;
        if (trade || !carry) {
          const int rb = c.vstar - (D - b);
          const int rs = c.vstar - Sb;
          if (trade && p == c.p_hi) sm.rem[0] = rb;
          if (trade && p == c.p_lo) sm.rem[1] = rs;
          if (carry) {
            nb = p > c.p_hi ? 0 : (p == c.p_hi ? b - rb : b);
            ns = p < c.p_lo ? 0 : (p == c.p_lo ? s - rs : s);
          } else {
            nb = ns = 0;
          }
        }
        D -= b;
        Sb += s;
        if constexpr (FEAT) {
          if (p > nl && p <= nl + 4) sm.feat[p - nl - 1] = ns;
          if (p < nl && p >= nl - 4) sm.feat[4 + nl - p - 1] = nb;
        }
        if (nb | ns) {
          rmin = min(rmin, p);
          rmax = max(rmax, p);
        }
        bv[i] = nb;
        sv[i] = ns;
      }
      if (trade || !carry) st_pairs<LTC>(book + 2 * p0, bv, sv);
    }
  } else {
    int D = D0, Sb = Sb0;
    for (int i = 0; i < LT; ++i) {
      const int p = p0 + i;
      if (p < pend) {
        const int b = book[2 * p], s = book[2 * p + 1];
        int nb = b, ns = s;
        if (trade || !carry) {
          const int rb = c.vstar - (D - b);
          const int rs = c.vstar - Sb;
          if (trade && p == c.p_hi) sm.rem[0] = rb;
          if (trade && p == c.p_lo) sm.rem[1] = rs;
          if (carry) {
            nb = p > c.p_hi ? 0 : (p == c.p_hi ? b - rb : b);
            ns = p < c.p_lo ? 0 : (p == c.p_lo ? s - rs : s);
          } else {
            nb = ns = 0;
          }
          book[2 * p] = nb;
          book[2 * p + 1] = ns;
        }
        D -= b;
        Sb += s;
        if constexpr (FEAT) {
          if (p > nl && p <= nl + 4) sm.feat[p - nl - 1] = ns;
          if (p < nl && p >= nl - 4) sm.feat[4 + nl - p - 1] = nb;
        }
        if (nb | ns) {
          rmin = min(rmin, p);
          rmax = max(rmax, p);
        }
      }
    }
  }
  {
    const int wmin = __reduce_min_sync(0xffffffffu, rmin);
    const int wmax = __reduce_max_sync(0xffffffffu, rmax);
    if (lane == 0 && wmax >= 0) {
      atomicMin(rng_next, wmin);
      atomicMax(rng_next + 1, wmax);
    }
  }
  if constexpr (FEAT) {
    if (t == 0) {
      // depth entries of ticks outside the region (or the grid) are zero
#pragma unroll
      for (int k = 1; k <= 4; ++k) {
        if (nl + k >= pend || nl + k < plo) sm.feat[k - 1] = 0;
        if (nl - k < plo || nl - k >= pend) sm.feat[4 + k - 1] = 0;
      }
    }
  }
  return c;
}

// Runs steps [s0, s0 + n_steps) of market m.  t: thread index in the group,
// bar: the group's barrier id, Lcap: the largest L the group's shared memory
// (sm) was carved for, REGACC: inventory and cash in registers (else in the
// shared-memory columns sm.inv / sm.cash).  CM: the book mode as a compile-time
// constant (0 discarded, 1 carried; the host launches such a kernel only for
// ensembles of that mode) or 2 (read from P.carry at run time).
template <int NT, int AK, bool AGGR, bool MLP, bool REGACC, bool FIT = false, int CM = 2>
__device__ void run_market(const DevParams& P, uint32_t m, uint32_t s0, uint32_t n_steps, const Smem& sm, int t,
                           int bar, int Lcap, MlpWG* mw = nullptr, const unsigned char* sw = nullptr) {
  static_assert(!(MLP && AGGR), "policy kernels use plain shared atomics");
  static_assert(!(MLP && REGACC), "policy rows read the inventory from shared memory");
  static_assert(!MLP || (NT >= 128 && NT % 128 == 0), "policy groups are whole warpgroups");
  static_assert((AK & (AK - 1)) == 0 && AK <= 32, "agents per thread: a power of two (agent = a0 ^ k)");
  const int lane = t & 31;
  const int wid = t >> 5;
  const int L = P.Ls ? P.Ls[m] : P.L_all;
  const int A = P.As ? P.As[m] : P.A_all;
  const int64_t aoff = P.agent_off ? P.agent_off[m] : (int64_t)m * (int64_t)P.A_all;
  if (A > NT * AK || L > Lcap || L < 2 || A < 0) {
    if (t == 0) atomicOr(P.err, ERR_SHAPE);
    return;  // uniform across the group
  }
  const int LT = (L + NT - 1) / NT;
  const int p0 = t * LT;
  // vector path when every owning thread has exactly LT in-grid ticks
  const int LTsel = ((LT == 1 || LT == 2 || LT == 4 || LT == 8) && (L % LT == 0)) ? LT : 0;
  int32_t* book = sm.book;
  const uint32_t book_s = (uint32_t)__cvta_generic_to_shared(book);

  // ---- load the market's state (128-bit accesses where aligned) -----------------
  uint32_t slot[AK];
  int inv[REGACC ? AK : 1];
  int cpend[REGACC ? AK : 1];  // cash since the last flush into sm.cash
  // FIT: the market's agents spread evenly over the group, akeff = ceil(A / NT)
  // of the AK slots per thread (a market smaller than the group's capacity then
  // takes fewer passes); else every thread owns AK agents.
  const int akeff = FIT ? min(AK, (A + NT - 1) / NT) : AK;
  const int a0 = t * akeff;
  const bool vec = (AK % 4 == 0) && ((aoff + a0) % 4 == 0) && (a0 + AK <= A) && akeff == AK;
  // 256-bit accesses: a thread's agents start on a 32-byte boundary of every array
  const bool wide = (AK % 8 == 0) && vec && ((aoff + a0) % 8 == 0);
  if constexpr (AK % 8 == 0) {
    if (wide) {
#pragma unroll
      for (int k = 0; k < AK; k += 8) {
        uint32_t sv[8], iv[8];
        int64_t c0[4], c1[4];
        ld_b32x8(P.slot + aoff + a0 + k, sv);
        ld_b32x8(P.inv + aoff + a0 + k, iv);
        ld_b64x4(P.cash + aoff + a0 + k, c0);
        ld_b64x4(P.cash + aoff + a0 + k + 4, c1);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          slot[k + i] = sv[i];
          if constexpr (REGACC)
            inv[k + i] = (int)iv[i];
          else
            sm.inv[(k + i) * NT + t] = (int)iv[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          sm.cash[(k + i) * NT + t] = c0[i];
          sm.cash[(k + 4 + i) * NT + t] = c1[i];
        }
      }
    }
  }
  if (wide) {
    // loaded above
  } else if (vec) {
#pragma unroll
    for (int k = 0; k < AK; k += 4) {
      const uint4 sv = *reinterpret_cast<const uint4*>(P.slot + aoff + a0 + k);
      const int4 iv = *reinterpret_cast<const int4*>(P.inv + aoff + a0 + k);
      const longlong2 c0 = *reinterpret_cast<const longlong2*>(P.cash + aoff + a0 + k);
      const longlong2 c1 = *reinterpret_cast<const longlong2*>(P.cash + aoff + a0 + k + 2);
      slot[k] = sv.x; slot[k + 1] = sv.y; slot[k + 2] = sv.z; slot[k + 3] = sv.w;
      if constexpr (REGACC) {
        inv[k] = iv.x; inv[k + 1] = iv.y; inv[k + 2] = iv.z; inv[k + 3] = iv.w;
      } else {
        sm.inv[(k + 0) * NT + t] = iv.x; sm.inv[(k + 1) * NT + t] = iv.y;
        sm.inv[(k + 2) * NT + t] = iv.z; sm.inv[(k + 3) * NT + t] = iv.w;
      }
      sm.cash[(k + 0) * NT + t] = c0.x; sm.cash[(k + 1) * NT + t] = c0.y;
      sm.cash[(k + 2) * NT + t] = c1.x; sm.cash[(k + 3) * NT + t] = c1.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < AK; ++k) {
      const int a = a0 + k;
      const bool v = a < A && k < akeff;
      slot[k] = v ? P.slot[aoff + a] : 0u;
      if constexpr (REGACC)
        inv[k] = v ? P.inv[aoff + a] : 0;
      else
        sm.inv[k * NT + t] = v ? P.inv[aoff + a] : 0;
      sm.cash[k * NT + t] = v ? P.cash[aoff + a] : 0ll;
    }
  }
  if constexpr (REGACC) {
#pragma unroll
    for (int k = 0; k < AK; ++k) cpend[k] = 0;
  }
  const int32_t* mi = P.mi32 + (size_t)m * MI32_STRIDE;
  int hist[KS_HISTORY];
#pragma unroll
  for (int j = 0; j < KS_HISTORY; ++j) hist[j] = mi[MI_HIST + j];
  int last = mi[MI_LAST];
  const int fund = mi[MI_FUND];
  int trades = mi[MI_TRADES];
  int lastv = mi[MI_LASTV];
  const int64_t* mi64 = P.mi64 + (size_t)m * MI64_STRIDE;
  int64_t sump = mi64[MI_SUMP];
  int64_t sumv = mi64[MI_SUMV];
  uint64_t hash = (uint64_t)mi64[MI_HASH];

  RuleConsts rc;
  rc.zi_off = P.zi_off;
  rc.zi_n = 2u * (uint32_t)P.zi_off + 1u;
  rc.zi_qmax = (uint32_t)P.zi_qmax;
  rc.mom_n = (uint32_t)P.mom_omax + 1u;
  rc.mr_n = (uint32_t)P.mr_omax + 1u;
  rc.rb_qmax = (uint32_t)P.rb_qmax;
  const uint32_t gm = P.market_base + m;
  // rule constants of the first step's orders
  StepRules sr0 = step_rules(P, s0, gm, hist[0], hist_at(hist, P.mom_lb), last, fund);
  if (t < 8) decision_row(sm.drow, sm.dsell, t, last, sr0.side_mom, sr0.side_mr, rc);

  // rebuild the aggregated resting book from the working orders
  for (int i = t; i < 2 * book_len(Lcap); i += NT) book[i] = 0;
  if (t < 8) sm.kx[t] = 0ull;
  if (t < 4) sm.rng[t] = (t & 1) ? -1 : 0x7FFFFFFF;
  gsync<NT>(bar);
#pragma unroll
  for (int k = 0; k < AK; ++k) {
    // an order word written through ks_write_state may name a tick outside the grid
    if (w_qty(slot[k]) != 0u && (int)w_tick(slot[k]) >= L) {
      atomicOr(P.err, ERR_TICK);
      slot[k] &= W_STATIC;
    }
    book_add<AGGR>(book_s, w_qty(slot[k]) != 0u, slot[k]);
  }

  static_assert(CM >= 0 && CM <= 2, "book mode: 0 discarded, 1 carried, 2 read at run time");
  const bool carry = CM == 2 ? P.carry != 0 : CM == 1;
  const uint32_t cthr = carry ? P.cancel_thr : 0u;     // a discarded book has nothing to cancel
  const uint32_t keep = carry ? 0xFFFFFFFFu : W_STATIC;  // what of an order word survives the step
  const bool traced = m < P.trace_markets;
  const bool tie1 = P.tie_rule == KS_TIE_MIN_IMBALANCE;

  const bool policy_on = MLP && P.mlp != nullptr && P.mlp_pct > 0;
  // every new order lies within dwin ticks of the last clearing tick
  const int dwin = max(max(P.zi_off, P.mom_omax), max(P.mr_omax, policy_on ? MLP_OFF_MAX : 0));
  const int blen = book_len(Lcap);
  StepFeat sf;
  if constexpr (MLP) {
    // the policy inputs of the first step read the rebuilt book
    gsync<NT>(bar);
    publish_depth(sm, book, L, last, p0, LT, t);
    gsync<NT>(bar);
#pragma unroll
    for (int j = 0; j < 8; ++j) sf.h[j] = hist[j] - hist[j + 1];
    sf.lastv = lastv;
    sf.depth = sm.feat;
  }

  // orders of the first step
  if (n_steps > 0) {
    const StepRules& sr = sr0;
    const uint32_t x0a = sr.sk.c0 ^ (uint32_t)a0;
    uint32_t pflags = 0;
#pragma unroll
    for (int k = 0; k < AK; ++k) {
      if (FIT && k >= akeff) break;
      const uint32_t x0 = FIT ? sr.sk.c0 ^ (uint32_t)(a0 + k) : x0a ^ (uint32_t)k;
      if constexpr (MLP) {
        bool pol = false;
        slot[k] = order_agent<AGGR, true>(slot[k], a0 + k, x0, a0 + k < A, sr, cthr, L, sm.drow, sm.dsell, book_s, P.rk, &pol,
                                          &P, &sf, sm.inv[k * NT + t]);
        pflags |= pol ? (1u << k) : 0u;
      } else {
        slot[k] = order_agent<AGGR, false, CM>(slot[k], a0 + k, x0, a0 + k < A, sr, cthr, L, sm.drow, sm.dsell, book_s, P.rk);
      }
    }
    if constexpr (MLP) {
      if (policy_on)
        policy_phase<NT, AK>(P, sm, *mw, sw, slot, pflags, t, bar, a0, A, L, s0, gm, sf, last, aoff, traced, book,
                             akeff);
    }
  }

  for (uint32_t j = 0; j < n_steps; ++j) {
    const uint32_t s = s0 + j;
    unsigned long long* kx = sm.kx + 4 * (j & 1);
    gsync<NT>(bar);  // B1: all orders of step s are in the book

    // ---- clearing and residual book ----------------------------------------------------
    unsigned long long* kx_next = sm.kx + 4 * ((j + 1) & 1);
    // The region to clear: after the first step of the call, only ticks
    // that can hold an order -- those that rested after the previous step
    // and the window of new orders around the last tick -- rounded to a
    // span of GT x {1, 2, 4, 8} ticks from a multiple of 8 (vector loads);
    // the whole grid when that span is not smaller.
    int plo = 0, pend = L, lts = LTsel, ltr = LT, p0r = p0;
    if (j > 0) {
      const int rlo = sm.rng[2 * (j & 1)], rhi = sm.rng[2 * (j & 1) + 1];
      const int lo = max(0, min(rlo, last - dwin)) & ~7;
      const int hi = min(L - 1, max(rhi, last + dwin));
      int lt = 1;
      while (lt < 8 && NT * lt < hi - lo + 1) lt <<= 1;
      const int span = NT * lt;
      if (span >= hi - lo + 1 && span <= blen && span < LT * NT) {
        plo = min(lo, blen - span);
        pend = plo + span;
        lts = lt;
        ltr = lt;
        p0r = plo + t * lt;
      }
    }
    if (t == 0) {  // range of the step after next (its last reader was the previous step)
      sm.rng[2 * ((j + 1) & 1)] = 0x7FFFFFFF;
      sm.rng[2 * ((j + 1) & 1) + 1] = -1;
    }
    int32_t* rng_next = sm.rng + 2 * ((j + 1) & 1);
    ClearOut c;
    switch (lts) {
      case 1: c = clear_step<NT, 1, MLP>(sm, book, L, ltr, p0r, plo, pend, t, bar, kx, kx_next, rng_next, tie1, carry, last); break;
      case 2: c = clear_step<NT, 2, MLP>(sm, book, L, ltr, p0r, plo, pend, t, bar, kx, kx_next, rng_next, tie1, carry, last); break;
      case 4: c = clear_step<NT, 4, MLP>(sm, book, L, ltr, p0r, plo, pend, t, bar, kx, kx_next, rng_next, tie1, carry, last); break;
      case 8: c = clear_step<NT, 8, MLP>(sm, book, L, ltr, p0r, plo, pend, t, bar, kx, kx_next, rng_next, tie1, carry, last); break;
      default: c = clear_step<NT, 0, MLP>(sm, book, L, ltr, p0r, plo, pend, t, bar, kx, kx_next, rng_next, tie1, carry, last); break;
    }
    const int vstar = c.vstar, pstar = c.pstar;
    const bool trade = vstar > 0;
    // An order of side/tick bits st fills fully when it is strictly better
    // than its side's marginal tick (rank > 0) and is rationed at it (rank
    // 0): rank = st - key_b for buys, key_s - st for sells.  Without a trade
    // the keys put every order below its margin.
    const uint32_t key_b = trade ? (uint32_t)c.p_hi << W_TICK_SHIFT : 0x1FFFFFFFu;
    const uint32_t key_s = trade ? (((uint32_t)c.p_lo << W_TICK_SHIFT) | W_SIDE) : 0u;

    // ---- marginal quantities in agent order --------------------------------------------
    uint32_t exB = 0, exS = 0;
    if (trade) {
      uint32_t mB = 0, mS = 0;
#pragma unroll
      for (int k = 0; k < AK; ++k) {
        if (FIT && k >= akeff) break;
        const uint32_t st = slot[k] & W_ST;
        const uint32_t q = w_qty(slot[k]);
        mB += st == key_b ? q : 0u;
        mS += st == key_s ? q : 0u;
      }
      uint32_t iB = mB, iS = mS;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t ob = __shfl_up_sync(0xffffffffu, iB, d);
        const uint32_t os = __shfl_up_sync(0xffffffffu, iS, d);
        if (lane >= d) { iB += ob; iS += os; }
      }
      if (lane == 31) { sm.wMB[wid] = iB; sm.wMS[wid] = iS; }
      exB = iB - mB;
      exS = iS - mS;
    }

    // ---- market scalars of step s ---------------------------------------------------------
    if (trade) last = pstar;
#pragma unroll
    for (int h = KS_HISTORY - 1; h > 0; --h) hist[h] = hist[h - 1];
    hist[0] = last;
    if (t == 0) {
      const int pt = trade ? pstar : -1;
      if (trade) {
        sump += pstar;
        trades += 1;
      }
      sumv += vstar;
      lastv = vstar;
      hash = trace_mix(hash, s, pt, vstar);
      if (traced && s < P.trace_steps) {
        int32_t* tr = P.trace + ((size_t)m * P.trace_steps + s) * 2;
        tr[0] = pt;
        tr[1] = vstar;
      }
    }
    const bool more = j + 1 < n_steps;
    const StepRules sr = step_rules(P, s + 1, gm, hist[0], hist_at(hist, P.mom_lb), last, fund);
    {
      // lanes 0-7 of warp 1 write the rows: warp 0 also carries the market
      // scalars before this barrier (0.8% on the 8192-market workload)
      constexpr int TR = NT >= 64 ? 32 : 0;
      if (t >= TR && t < TR + 8) decision_row(sm.drow, sm.dsell, t - TR, last, sr.side_mom, sr.side_mr, rc);
    }
    gsync<NT>(bar);  // B5: book residual, remainders, marginal totals and rule constants visible

    // ---- fills of step s, fused with the orders of step s+1 ------------------------------
    const uint32_t x0a = sr.sk.c0 ^ (uint32_t)a0;
    if constexpr (MLP) {
#pragma unroll
      for (int q = 0; q < 8; ++q) sf.h[q] = hist[q] - hist[q + 1];
      sf.lastv = vstar;
    }
    // units still to fill at the marginal buy / sell tick before my first agent
    int remB = 0, remS = 0;
    if (trade) {
      remB = sm.rem[0] - (int)(exB + __reduce_add_sync(0xffffffffu, lane < wid ? sm.wMB[lane] : 0u));
      remS = sm.rem[1] - (int)(exS + __reduce_add_sync(0xffffffffu, lane < wid ? sm.wMS[lane] : 0u));
    }
    uint32_t pflags = 0;
    // The orders of several agents share one block (their Philox chains
    // interleave): four in the plain kernel (+0.8% over two, +5% over one),
    // two in the batched kernel, whose agents spread unevenly over the
    // group's slots (four was 3% slower there); the policy kernels cannot
    // spare the registers.
    constexpr int IL = (AK < 2 || MLP) ? 1 : ((FIT || AK < 4) ? 2 : 4);
#pragma unroll
    for (int kb = 0; kb < AK; kb += IL) {
      if (FIT && kb >= akeff) break;
      uint32_t sl[IL];
#pragma unroll
      for (int i = 0; i < IL; ++i) {
        const int k = kb + i;
        const uint32_t sl0 = slot[k];
        const int q = (int)w_qty(sl0);
        const uint32_t st = sl0 & W_ST;
        const bool sell = (sl0 & W_SIDE) != 0u;
        const int rank = sell ? (int)(key_s - st) : (int)(st - key_b);
        int f = rank > 0 ? q : 0;
        if constexpr (CM != 2) {
          // rationed at the marginal tick, in agent order: few orders sit
          // there, so a warp vote skips the rule in most warps (with the book
          // mode fixed at compile time, 1.1% on the 8192-market workload)
          if (__any_sync(0xffffffffu, rank == 0)) {
            const bool marg = rank == 0;
            const int fm = min(max(sell ? remS : remB, 0), q);
            f = marg ? fm : f;
            const int adv = marg ? q : 0;
            remS -= sell ? adv : 0;
            remB -= sell ? 0 : adv;
          }
        } else if (rank == 0) {
          // rationed at the marginal tick, in agent order (few orders sit there)
          if (sell) {
            f = min(max(remS, 0), q);
            remS -= q;
          } else {
            f = min(max(remB, 0), q);
            remB -= q;
          }
        }
        const int sfill = sell ? -f : f;
        if constexpr (REGACC) {
          inv[k] += sfill;
          cpend[k] -= pstar * sfill;
        } else if (f) {
          sm.inv[k * NT + t] += sfill;
          sm.cash[k * NT + t] -= (int64_t)pstar * sfill;
        }
        sl[i] = (sl0 - (uint32_t)f) & keep;
      }
      if (more) {
#pragma unroll
        for (int i = 0; i < IL; ++i) {
          const int k = kb + i;
          const uint32_t x0 = FIT ? sr.sk.c0 ^ (uint32_t)(a0 + k) : x0a ^ (uint32_t)k;
          const bool valid = a0 + k < A && (!FIT || k < akeff);
          if constexpr (MLP) {
            bool pol = false;
            sl[i] = order_agent<AGGR, true>(sl[i], a0 + k, x0, valid, sr, cthr, L, sm.drow, sm.dsell, book_s, P.rk, &pol, &P,
                                            &sf, sm.inv[k * NT + t]);
            pflags |= pol ? (1u << k) : 0u;
          } else {
            sl[i] = order_agent<AGGR, false, CM>(sl[i], a0 + k, x0, valid, sr, cthr, L, sm.drow, sm.dsell, book_s, P.rk);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < IL; ++i) slot[kb + i] = sl[i];
    }
    if constexpr (REGACC) {
      if ((j + 1) % CASH_FLUSH_STEPS == 0) {
#pragma unroll
        for (int k = 0; k < AK; ++k) {
          sm.cash[k * NT + t] += cpend[k];
          cpend[k] = 0;
        }
      }
    }
    if constexpr (MLP) {
      if (policy_on && more)
        policy_phase<NT, AK>(P, sm, *mw, sw, slot, pflags, t, bar, a0, A, L, s + 1, gm, sf, last, aoff, traced,
                             book, akeff);
    }
  }

  // ---- store ---------------------------------------------------------------------------
  if constexpr (AK % 8 == 0) {
    if (wide) {
#pragma unroll
      for (int k = 0; k < AK; k += 8) {
        uint32_t sv[8], iv[8];
        int64_t c0[4], c1[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          sv[i] = slot[k + i];
          if constexpr (REGACC)
            iv[i] = (uint32_t)inv[k + i];
          else
            iv[i] = (uint32_t)sm.inv[(k + i) * NT + t];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          c0[i] = sm.cash[(k + i) * NT + t];
          c1[i] = sm.cash[(k + 4 + i) * NT + t];
          if constexpr (REGACC) {
            c0[i] += cpend[k + i];
            c1[i] += cpend[k + 4 + i];
          }
        }
        st_b32x8(P.slot + aoff + a0 + k, sv);
        st_b32x8(P.inv + aoff + a0 + k, iv);
        st_b64x4(P.cash + aoff + a0 + k, c0);
        st_b64x4(P.cash + aoff + a0 + k + 4, c1);
      }
    }
  }
  if (wide) {
    // stored above
  } else if (vec) {
#pragma unroll
    for (int k = 0; k < AK; k += 4) {
      *reinterpret_cast<uint4*>(P.slot + aoff + a0 + k) = make_uint4(slot[k], slot[k + 1], slot[k + 2], slot[k + 3]);
      longlong2 c0, c1;
      c0.x = sm.cash[(k + 0) * NT + t];
      c0.y = sm.cash[(k + 1) * NT + t];
      c1.x = sm.cash[(k + 2) * NT + t];
      c1.y = sm.cash[(k + 3) * NT + t];
      if constexpr (REGACC) {
        *reinterpret_cast<int4*>(P.inv + aoff + a0 + k) = make_int4(inv[k], inv[k + 1], inv[k + 2], inv[k + 3]);
        c0.x += cpend[k];
        c0.y += cpend[k + 1];
        c1.x += cpend[k + 2];
        c1.y += cpend[k + 3];
      } else {
        *reinterpret_cast<int4*>(P.inv + aoff + a0 + k) =
            make_int4(sm.inv[(k + 0) * NT + t], sm.inv[(k + 1) * NT + t], sm.inv[(k + 2) * NT + t],
                      sm.inv[(k + 3) * NT + t]);
      }
      *reinterpret_cast<longlong2*>(P.cash + aoff + a0 + k) = c0;
      *reinterpret_cast<longlong2*>(P.cash + aoff + a0 + k + 2) = c1;
    }
  } else {
#pragma unroll
    for (int k = 0; k < AK; ++k) {
      const int a = a0 + k;
      if (a < A && k < akeff) {
        P.slot[aoff + a] = slot[k];
        if constexpr (REGACC) {
          P.inv[aoff + a] = inv[k];
          P.cash[aoff + a] = sm.cash[k * NT + t] + cpend[k];
        } else {
          P.inv[aoff + a] = sm.inv[k * NT + t];
          P.cash[aoff + a] = sm.cash[k * NT + t];
        }
      }
    }
  }
  if (t == 0) {
    int32_t* mo = P.mi32 + (size_t)m * MI32_STRIDE;
    mo[MI_LAST] = last;
#pragma unroll
    for (int j = 0; j < KS_HISTORY; ++j) mo[MI_HIST + j] = hist[j];
    mo[MI_TRADES] = trades;
    mo[MI_LASTV] = lastv;
    int64_t* m64 = P.mi64 + (size_t)m * MI64_STRIDE;
    m64[MI_SUMP] = sump;
    m64[MI_SUMV] = sumv;
    m64[MI_HASH] = (int64_t)hash;
  }
  gsync<NT>(bar);  // shared memory is reused by the group's next market
}

}  // namespace ks
