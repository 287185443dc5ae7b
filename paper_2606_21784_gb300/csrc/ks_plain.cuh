// ks_plain.cuh -- persistent block-per-market call-auction kernel (sm_103a).
//
// One CTA owns one market at a time and keeps it on chip for all n steps of a
// call (the paper's Algorithm 1 and Sec. III-B residency, re-shaped for
// GB300): thread t owns agents [t*AK, t*AK+AK) in registers (order words) and
// shared memory (inventory, cash), and ticks [t*LT, t*LT+LT) of the
// aggregated book in shared memory.  Per step:
//   A  cancel + decide + shared atomics into BUY/SELL          (Alg. 1, Phase 3)
//   B  suffix scan of BUY and prefix scan of SELL by per-thread serial sums,
//      warp shuffles and one cross-warp pass; V = min(D_cum, S_cum) and two
//      packed max-reductions giving the lowest and the highest maximiser of V
//      (Eq. 1-2, Phase 4)
//   C  fills: buys above the highest maximiser and sells below the lowest fill
//      fully; the marginal ticks are rationed in agent order with one block
//      scan; residual book updated per tick without atomics        (Phase 5)
// Four CTA barriers per step; global memory is touched only at market load
// and store, so traffic does not grow with the number of steps.
#pragma once

#include <stdint.h>

#include "ks_device.cuh"

namespace ks {

struct Smem {
  int64_t* cash;  // [AK][NT]  (thread-private columns)
  int32_t* inv;   // [AK][NT]
  int32_t* buy;   // [book_len(Lmax)]
  int32_t* sell;  // [book_len(Lmax)]
  uint64_t* wLo;  // [32] warp partials
  uint64_t* wHi;
  uint64_t* wT;
  uint64_t* wM;
  int32_t* wD;
  int32_t* wS;
};

__host__ __device__ inline size_t plain_smem_layout(int nt, int ak, int Lmax, size_t* o) {
  size_t off = 0;
  o[0] = off; off += (size_t)8 * ak * nt;           // cash
  o[1] = off; off += (size_t)8 * 32 * 4;            // wLo, wHi, wT, wM
  o[2] = off; off += (size_t)4 * ak * nt;           // inv
  o[3] = off; off += (size_t)4 * book_len(Lmax);    // buy
  o[4] = off; off += (size_t)4 * book_len(Lmax);    // sell
  o[5] = off; off += (size_t)4 * 32 * 2;            // wD, wS
  return (off + 15) & ~(size_t)15;
}

template <int NT, int AK>
__device__ __forceinline__ Smem carve(unsigned char* raw, int Lmax) {
  size_t o[6];
  plain_smem_layout(NT, AK, Lmax, o);
  Smem s;
  s.cash = reinterpret_cast<int64_t*>(raw + o[0]);
  s.wLo = reinterpret_cast<uint64_t*>(raw + o[1]);
  s.wHi = s.wLo + 32;
  s.wT = s.wLo + 64;
  s.wM = s.wLo + 96;
  s.inv = reinterpret_cast<int32_t*>(raw + o[2]);
  s.buy = reinterpret_cast<int32_t*>(raw + o[3]);
  s.sell = reinterpret_cast<int32_t*>(raw + o[4]);
  s.wD = reinterpret_cast<int32_t*>(raw + o[5]);
  s.wS = s.wD + 32;
  return s;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    uint64_t o = __shfl_xor_sync(0xffffffffu, v, d);
    v = o > v ? o : v;
  }
  return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

__device__ __forceinline__ int warp_sum_i32(int v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Add q at (side, tick) of the book.  With AGGR, lanes of the warp holding the
// same (side, tick) first combine their quantities (__match_any_sync +
// __reduce_add_sync) and one lane issues the shared atomic.
template <bool AGGR>
__device__ __forceinline__ void book_add(const Smem& sm, bool valid, uint32_t sell, uint32_t tick, int q) {
  if constexpr (AGGR) {
    uint32_t key = valid ? ((sell << 12) | tick) : 0xFFFFFFFFu;
    unsigned peers = __match_any_sync(0xffffffffu, key);
    int tot = (int)__reduce_add_sync(peers, (unsigned)q);
    int leader = __ffs(peers) - 1;
    if (valid && (int)(threadIdx.x & 31) == leader) atomicAdd((sell ? sm.sell : sm.buy) + book_idx(tick), tot);
  } else {
    if (valid) atomicAdd((sell ? sm.sell : sm.buy) + book_idx(tick), q);
  }
}

template <int NT, int AK, bool AGGR>
__device__ void run_market(const DevParams& P, uint32_t m, uint32_t s0, uint32_t n_steps, const Smem& sm) {
  constexpr int NW = NT / 32;
  const int t = threadIdx.x;
  const int lane = t & 31;
  const int wid = t >> 5;
  const int L = P.Ls ? P.Ls[m] : P.L_all;
  const int A = P.As ? P.As[m] : P.A_all;
  const int64_t aoff = P.agent_off ? P.agent_off[m] : (int64_t)m * (int64_t)P.A_all;
  if (A > NT * AK || L > P.Lmax || L < 2 || A < 0) {
    if (t == 0) atomicOr(P.err, ERR_SHAPE);
    return;  // uniform across the CTA
  }
  const int LT = (L + NT - 1) / NT;
  const int p0 = t * LT;

  // ---- S0: load the market's state ------------------------------------------------
  uint32_t slot[AK];
#pragma unroll
  for (int k = 0; k < AK; ++k) {
    const int a = t * AK + k;
    const bool v = a < A;
    slot[k] = v ? P.slot[aoff + a] : 0u;
    sm.inv[k * NT + t] = v ? P.inv[aoff + a] : 0;
    sm.cash[k * NT + t] = v ? P.cash[aoff + a] : 0ll;
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

  // rebuild the aggregated resting book from the working orders
  const int blen = book_len(L);
  for (int i = t; i < blen; i += NT) {
    sm.buy[i] = 0;
    sm.sell[i] = 0;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < AK; ++k) {
    // an order word written through ks_write_state may name a tick outside the grid
    if (w_qty(slot[k]) != 0u && (int)w_tick(slot[k]) >= L) {
      atomicOr(P.err, ERR_TICK);
      slot[k] &= W_STATIC;
    }
    const uint32_t q = w_qty(slot[k]);
    book_add<AGGR>(sm, q != 0u, w_sell(slot[k]), w_tick(slot[k]), (int)q);
  }

  RuleConsts rc;
  rc.zi_off = P.zi_off;
  rc.zi_n = 2u * (uint32_t)P.zi_off + 1u;
  rc.zi_qmax = (uint32_t)P.zi_qmax;
  rc.mom_n = (uint32_t)P.mom_omax + 1u;
  rc.mr_n = (uint32_t)P.mr_omax + 1u;
  rc.rb_qmax = (uint32_t)P.rb_qmax;
  const bool carry = P.carry != 0;
  const uint32_t cthr = P.cancel_thr;
  const bool traced = m < P.trace_markets;

  for (uint32_t j = 0; j < n_steps; ++j) {
    const uint32_t s = s0 + j;
    // ---- A: cancellations and new orders ------------------------------------------
    const StepKey sk = step_key(s, P.market_base + m, 0u, P.key0, P.key1);
    int hlb = hist[1];
#pragma unroll
    for (int h = 2; h < KS_HISTORY; ++h) hlb = (P.mom_lb == h) ? hist[h] : hlb;
    const int ret = hist[0] - hlb;
    const int side_mom = ret > 0 ? 0 : (ret < 0 ? 1 : -1);
    const int side_mr = last < fund ? 0 : (last > fund ? 1 : -1);
#pragma unroll
    for (int k = 0; k < AK; ++k) {
      const int a = t * AK + k;
      const bool valid = a < A;
      const uint4 w = step_draw(sk, (uint32_t)a);
      uint32_t sl = slot[k];
      const uint32_t q = w_qty(sl);
      const bool cancel = valid && carry && q != 0u && w.x < cthr;
      if (cancel) atomicSub((w_sell(sl) ? sm.sell : sm.buy) + book_idx(w_tick(sl)), (int)q);
      const bool dec = valid && (q == 0u || cancel) && !(sl & W_MLP);
      const uint32_t ns = decide_rule(sl, w, last, side_mom, side_mr, L, rc);
      sl = dec ? ns : (cancel ? (sl & W_STATIC) : sl);
      book_add<AGGR>(sm, dec, w_sell(ns), w_tick(ns), (int)w_qty(ns));
      slot[k] = sl;
    }
    __syncthreads();  // B1: all orders of step s are in the book

    // ---- B: scans, V = min(D, S), lowest / highest maximiser ----------------------
    int sumB = 0, sumS = 0;
    for (int i = 0; i < LT; ++i) {
      const int p = p0 + i;
      if (p < L) {
        sumB += sm.buy[book_idx(p)];
        sumS += sm.sell[book_idx(p)];
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
    __syncthreads();  // B2
    {
      const int dw = (lane < NW && lane > wid) ? sm.wD[lane] : 0;
      const int sw = (lane < NW && lane < wid) ? sm.wS[lane] : 0;
      const int offD = warp_sum_i32(dw);
      const int offS = warp_sum_i32(sw);
      int D = offD + sufB;              // D_cum at my first tick
      int Sb = offS + preS - sumS;      // S_cum just below my first tick
      uint64_t kLo = 0, kHi = 0, kT = 0;
      const bool tie1 = P.tie_rule == KS_TIE_MIN_IMBALANCE;
      for (int i = 0; i < LT; ++i) {
        const int p = p0 + i;
        if (p < L) {
          const int b = sm.buy[book_idx(p)];
          const int sv = sm.sell[book_idx(p)];
          const int S = Sb + sv;
          const int v = min(D, S);
          const int Da = D - b;  // D_cum[p+1]
          const uint64_t vv = (uint64_t)(uint32_t)v << 40;
          const uint64_t lo = vv | ((uint64_t)(4095 - p) << 28) | (uint64_t)(uint32_t)Sb;
          const uint64_t hi = vv | ((uint64_t)p << 28) | (uint64_t)(uint32_t)Da;
          kLo = lo > kLo ? lo : kLo;
          kHi = hi > kHi ? hi : kHi;
          if (tie1) {
            const int imb = min(abs(D - S), 0x0FFFFFFF);
            const uint64_t tk = vv | ((uint64_t)(0x0FFFFFFF - imb) << 12) | (uint64_t)(4095 - p);
            kT = tk > kT ? tk : kT;
          }
          D = Da;
          Sb = S;
        }
      }
      kLo = warp_max_u64(kLo);
      kHi = warp_max_u64(kHi);
      if (tie1) kT = warp_max_u64(kT);
      if (lane == 0) {
        sm.wLo[wid] = kLo;
        sm.wHi[wid] = kHi;
        sm.wT[wid] = kT;
      }
    }
    __syncthreads();  // B3
    uint64_t kLo = lane < NW ? sm.wLo[lane] : 0ull;
    uint64_t kHi = lane < NW ? sm.wHi[lane] : 0ull;
    kLo = warp_max_u64(kLo);
    kHi = warp_max_u64(kHi);
    const int vstar = (int)(kLo >> 40);
    const int p_lo = 4095 - (int)((kLo >> 28) & 4095u);
    const int p_hi = (int)((kHi >> 28) & 4095u);
    const int R_s = vstar - (int)(kLo & 0x0FFFFFFFu);  // units sold at the marginal sell tick
    const int R_b = vstar - (int)(kHi & 0x0FFFFFFFu);  // units bought at the marginal buy tick
    int pstar = p_lo;
    if (P.tie_rule == KS_TIE_MIN_IMBALANCE) {
      uint64_t kT = lane < NW ? sm.wT[lane] : 0ull;
      kT = warp_max_u64(kT);
      pstar = 4095 - (int)(kT & 4095u);
    }
    const bool trade = vstar > 0;

    // residual book, per tick and without atomics (Phase 5)
    if (carry) {
      if (trade) {
        for (int i = 0; i < LT; ++i) {
          const int p = p0 + i;
          if (p < L) {
            if (p > p_hi) sm.buy[book_idx(p)] = 0;
            else if (p == p_hi) sm.buy[book_idx(p)] -= R_b;
            if (p < p_lo) sm.sell[book_idx(p)] = 0;
            else if (p == p_lo) sm.sell[book_idx(p)] -= R_s;
          }
        }
      }
    } else {
      for (int i = 0; i < LT; ++i) {
        const int p = p0 + i;
        if (p < L) {
          sm.buy[book_idx(p)] = 0;
          sm.sell[book_idx(p)] = 0;
        }
      }
    }

    // ---- C: fills ------------------------------------------------------------------
    uint64_t mine = 0;
    if (trade) {
      uint32_t mB = 0, mS = 0;
#pragma unroll
      for (int k = 0; k < AK; ++k) {
        const uint32_t sl = slot[k];
        const uint32_t q = w_qty(sl);
        const int tk = (int)w_tick(sl);
        if (q && !w_sell(sl) && tk == p_hi) mB += q;
        if (q && w_sell(sl) && tk == p_lo) mS += q;
      }
      mine = ((uint64_t)mS << 32) | (uint64_t)mB;
      uint64_t inc = mine;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
      }
      if (lane == 31) sm.wM[wid] = inc;
      mine = inc - mine;  // exclusive within the warp
    }
    __syncthreads();  // B5 (also orders the residual-book writes before step s+1)
    if (trade) {
      const uint64_t wo = warp_sum_u64((lane < NW && lane < wid) ? sm.wM[lane] : 0ull);
      const uint64_t ex = mine + wo;
      int preB = (int)(uint32_t)ex;
      int preSl = (int)(uint32_t)(ex >> 32);
#pragma unroll
      for (int k = 0; k < AK; ++k) {
        uint32_t sl = slot[k];
        const int q = (int)w_qty(sl);
        const int tk = (int)w_tick(sl);
        const bool sell = w_sell(sl) != 0u;
        int f = 0;
        if (q) {
          if (!sell) {
            if (tk > p_hi) f = q;
            else if (tk == p_hi) { f = min(max(R_b - preB, 0), q); preB += q; }
          } else {
            if (tk < p_lo) f = q;
            else if (tk == p_lo) { f = min(max(R_s - preSl, 0), q); preSl += q; }
          }
        }
        if (f) {
          sm.inv[k * NT + t] += sell ? -f : f;
          sm.cash[k * NT + t] += sell ? (int64_t)pstar * f : -(int64_t)pstar * f;
          sl -= (uint32_t)f;
        }
        slot[k] = sl;
      }
    }
    if (!carry) {
#pragma unroll
      for (int k = 0; k < AK; ++k) slot[k] &= W_STATIC;
    }

    // ---- market scalars ------------------------------------------------------------
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
  }

  // ---- S8: store ------------------------------------------------------------------------
#pragma unroll
  for (int k = 0; k < AK; ++k) {
    const int a = t * AK + k;
    if (a < A) {
      P.slot[aoff + a] = slot[k];
      P.inv[aoff + a] = sm.inv[k * NT + t];
      P.cash[aoff + a] = sm.cash[k * NT + t];
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
  __syncthreads();  // shared memory is reused by the CTA's next market
}

template <int NT, int AK, bool AGGR>
__global__ void __launch_bounds__(NT) plain_kernel(DevParams P, uint32_t n_steps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem sm = carve<NT, AK>(smem_raw, P.Lmax);
  const uint32_t s0 = (uint32_t)(*P.step);
  for (uint32_t m = blockIdx.x; m < P.M; m += gridDim.x) run_market<NT, AK, AGGR>(P, m, s0, n_steps, sm);
}

template <int NT, int AK>
cudaError_t launch_plain(const DevParams& p, uint32_t n_steps, int grid, size_t smem, cudaStream_t st,
                         int aggregate) {
  if (aggregate) {
    plain_kernel<NT, AK, true><<<grid, NT, smem, st>>>(p, n_steps);
  } else {
    plain_kernel<NT, AK, false><<<grid, NT, smem, st>>>(p, n_steps);
  }
  return cudaGetLastError();
}

}  // namespace ks
