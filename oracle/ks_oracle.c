/*
 * ks_oracle.c -- plain, slow, single-threaded CPU oracle of persistent
 * call-auction clearing over an ensemble of independent markets.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load or call this file.  It shares no code,
 * header, table or helper with the CUDA library: every constant below is
 * restated here from its published source.
 *
 * What it computes, and where each piece comes from:
 *  - Clearing (Sec. II-A, Eq. 1-2): D_cum[p] = sum_{q>=p} BUY[q],
 *    S_cum[p] = sum_{q<=p} SELL[q], V(p) = min(D_cum, S_cum),
 *    p* = argmax V with ties to the lowest tick (Sec. III-D, Phase 4).
 *    With max V = 0 there is no trade (a reading: the paper is silent).
 *  - Allocation (Sec. IV-C worked example): all trades at p*; buys fill in
 *    price priority from the top tick down, sells from the bottom tick up,
 *    until V* is used up on each side.  Inside one tick the orders fill in
 *    ascending agent index (a reading: the paper's book has no order identity).
 *  - Agents, RNG and book dynamics follow the stated readings of the
 *    benchmark configurations (one working order per agent, Philox4x32-10
 *    draws keyed by (seed, market, agent, step)); see the function comments.
 *  - Philox4x32-10 is written from Salmon, Moraes, Dror and Shaw, "Parallel
 *    random numbers: as easy as 1, 2, 3", SC'11.
 *  - The trace hash uses the SplitMix64 finaliser printed in Sec. III-G.
 *  - The MLP policy (32 -> 64 -> 64 -> 3 side + 33 offset + 1 log-qty logits,
 *    ReLU) forward and backward are plain fp64 loops; the behaviour-cloning
 *    loss is cross-entropy on side and offset plus squared error on
 *    log-quantity.  Features, sampling and the loss are readings
 *    of the learned-agent configuration (the paper has no learned agents).
 *
 * The clearing loops are the definitions evaluated directly; the allocation is
 * a greedy walk over price levels.  No blocking, fusion or reordering.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): round function on a 4x32 counter with a 2x32 key.  */
/* Multipliers and Weyl key increments as published with the generator.     */
/* ------------------------------------------------------------------------ */
static const uint32_t KO_PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t KO_PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t KO_PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t KO_PHILOX_WEYL_B = 0xBB67AE85u;

void ko_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* key schedule: bump before every round but the first */
      k0 += KO_PHILOX_WEYL_A;
      k1 += KO_PHILOX_WEYL_B;
    }
    uint64_t prodA = (uint64_t)KO_PHILOX_MUL_A * (uint64_t)x0;
    uint64_t prodB = (uint64_t)KO_PHILOX_MUL_B * (uint64_t)x2;
    uint32_t hiA = (uint32_t)(prodA >> 32), loA = (uint32_t)prodA;
    uint32_t hiB = (uint32_t)(prodB >> 32), loB = (uint32_t)prodB;
    uint32_t y0 = hiB ^ x1 ^ k0;
    uint32_t y1 = loB;
    uint32_t y2 = hiA ^ x3 ^ k1;
    uint32_t y3 = loA;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One Philox block for counter (step, agent, market, stream) under the key   */
/* (seed low word, seed high word).                                           */
static void ko_draw(uint64_t seed, uint32_t step, uint32_t agent, uint32_t market,
                    uint32_t stream, uint32_t w[4]) {
  uint32_t ctr[4] = {step, agent, market, stream};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  ko_philox4x32_10(ctr, key, w);
}

/* floor(u * n) for u = w / 2^32: the integer range draw of Sec. III-C's      */
/* q = 1 + floor(u q_max), taken on the 32-bit word directly.                 */
static int64_t ko_range(uint32_t w, int64_t n) { return (int64_t)(((uint64_t)w * (uint64_t)n) >> 32); }

static int32_t ko_clamp(int64_t x, int32_t lo, int32_t hi) {
  if (x < lo) return lo;
  if (x > hi) return hi;
  return (int32_t)x;
}

/* SplitMix64 finaliser (Sec. III-G) used to fold the clearing trace. */
static uint64_t ko_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

uint64_t ko_trace_hash_update(uint64_t h, uint32_t step, int32_t pstar, int32_t vol) {
  uint64_t word = ((uint64_t)(uint32_t)pstar << 32) | (uint64_t)(uint32_t)vol;
  return ko_mix64(h ^ word ^ ((uint64_t)step * 0x9E3779B97F4A7C15ull));
}

/* ------------------------------------------------------------------------ */
/* Clearing of one aggregated book (Sec. II-A, Eq. 1-2; Sec. III-D).          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t vstar;   /* executed volume V* = max_p V(p); 0 means no trade     */
  int32_t pstar;   /* clearing tick, -1 when V* = 0                         */
  int32_t p_buy;   /* marginal buy tick  max{p : D_cum[p] >= V*}, -1 if none */
  int32_t p_sell;  /* marginal sell tick min{p : S_cum[p] >= V*}, -1 if none */
  int32_t argmax;  /* argmax of V under the tie rule, defined also at V* = 0 */
} ko_clear_result;

/* tie_rule 0: lowest tick among maximisers (Sec. III-D).
 * tie_rule 1: smallest |D_cum - S_cum| among maximisers, then lowest tick.   */
int ko_clear_book(int32_t L, const int64_t* buy, const int64_t* sell, int32_t tie_rule,
                  int64_t* dcum, int64_t* scum, int64_t* vol, ko_clear_result* res) {
  if (L <= 0) return -1;
  /* D_cum[p] = sum over q >= p of BUY[q] */
  int64_t run = 0;
  for (int32_t p = L - 1; p >= 0; --p) {
    run += buy[p];
    dcum[p] = run;
  }
  /* S_cum[p] = sum over q <= p of SELL[q] */
  run = 0;
  for (int32_t p = 0; p < L; ++p) {
    run += sell[p];
    scum[p] = run;
  }
  /* V(p) = min(D_cum[p], S_cum[p]) */
  for (int32_t p = 0; p < L; ++p) vol[p] = dcum[p] < scum[p] ? dcum[p] : scum[p];
  /* maximum executable volume */
  int64_t vmax = vol[0];
  for (int32_t p = 1; p < L; ++p)
    if (vol[p] > vmax) vmax = vol[p];
  /* clearing tick under the tie rule */
  int32_t best = -1;
  for (int32_t p = 0; p < L; ++p) {
    if (vol[p] != vmax) continue;
    if (best < 0) { best = p; continue; }
    if (tie_rule == 1) {
      int64_t ib = dcum[best] - scum[best]; if (ib < 0) ib = -ib;
      int64_t ip = dcum[p] - scum[p];       if (ip < 0) ip = -ip;
      if (ip < ib) best = p;               /* equal imbalance keeps the lower tick */
    }
  }
  res->argmax = best;
  res->vstar = vmax;
  if (vmax <= 0) {
    res->vstar = 0;
    res->pstar = -1;
    res->p_buy = -1;
    res->p_sell = -1;
    return 0;
  }
  res->pstar = best;
  res->p_buy = -1;
  for (int32_t p = 0; p < L; ++p)
    if (dcum[p] >= vmax) res->p_buy = p;      /* keeps the largest such p */
  res->p_sell = -1;
  for (int32_t p = L - 1; p >= 0; --p)
    if (scum[p] >= vmax) res->p_sell = p;     /* keeps the smallest such p */
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Greedy allocation (Sec. IV-C): fill buys from the highest tick down and    */
/* sells from the lowest tick up, each tick in ascending agent index, until   */
/* V* is used up on each side.  side: 0 = buy, 1 = sell; qty 0 = no order.   */
/* fill[a] receives the executed quantity of agent a's order.                 */
/* ------------------------------------------------------------------------ */
int ko_allocate(int32_t L, int32_t A, const int32_t* side, const int32_t* tick,
                const int32_t* qty, int64_t vstar, int32_t* fill) {
  for (int32_t a = 0; a < A; ++a) fill[a] = 0;
  if (vstar <= 0) return 0;
  /* per-tick order lists in ascending agent index: count, then place */
  int32_t* start = (int32_t*)calloc((size_t)2 * (L + 1), sizeof(int32_t));
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A > 0 ? A : 1));
  int32_t* cursor = (int32_t*)malloc(sizeof(int32_t) * (size_t)2 * L);
  if (!start || !order || !cursor) { free(start); free(order); free(cursor); return -2; }
  for (int32_t a = 0; a < A; ++a) {
    if (qty[a] <= 0) continue;
    if (tick[a] < 0 || tick[a] >= L) { free(start); free(order); free(cursor); return -3; }
    start[side[a] * (L + 1) + tick[a] + 1] += 1;
  }
  int32_t base = 0;
  for (int32_t s = 0; s < 2; ++s) {
    start[s * (L + 1)] = base;
    for (int32_t p = 0; p < L; ++p) {
      int32_t c = start[s * (L + 1) + p + 1];
      start[s * (L + 1) + p + 1] = start[s * (L + 1) + p] + c;
    }
    base = start[s * (L + 1) + L];
  }
  for (int32_t s = 0; s < 2; ++s)
    for (int32_t p = 0; p < L; ++p) cursor[s * L + p] = start[s * (L + 1) + p];
  for (int32_t a = 0; a < A; ++a) {
    if (qty[a] <= 0) continue;
    order[cursor[side[a] * L + tick[a]]++] = a;
  }
  /* buys: highest tick first */
  int64_t left = vstar;
  for (int32_t p = L - 1; p >= 0 && left > 0; --p) {
    for (int32_t i = start[p]; i < start[p + 1] && left > 0; ++i) {
      int32_t a = order[i];
      int64_t f = qty[a] < left ? qty[a] : left;
      fill[a] = (int32_t)f;
      left -= f;
    }
  }
  int64_t buy_left = left;
  /* sells: lowest tick first */
  left = vstar;
  for (int32_t p = 0; p < L && left > 0; ++p) {
    for (int32_t i = start[(L + 1) + p]; i < start[(L + 1) + p + 1] && left > 0; ++i) {
      int32_t a = order[i];
      int64_t f = qty[a] < left ? qty[a] : left;
      fill[a] = (int32_t)f;
      left -= f;
    }
  }
  free(start); free(order); free(cursor);
  /* V* never exceeds either side's total, so both walks must finish */
  return (buy_left == 0 && left == 0) ? 0 : -4;
}


/* ------------------------------------------------------------------------ */
/* MLP policy (fp64).  Parameter vector layout:                              */
/*   W1[64][32], b1[64], W2[64][64], b2[64], W3[37][64], b3[37].            */
/* ------------------------------------------------------------------------ */
#define KO_IN 32
#define KO_H 64
#define KO_OUT 37
#define KO_NSIDE 3
#define KO_NOFF 33
#define KO_OFF_MAX 16
#define KO_NPARAM (KO_H * KO_IN + KO_H + KO_H * KO_H + KO_H + KO_OUT * KO_H + KO_OUT)
#define KO_NRAW 18

int32_t ko_mlp_nparam(void) { return KO_NPARAM; }

typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
} ko_mlp_view;

static ko_mlp_view ko_mlp_split(const double* w) {
  ko_mlp_view v;
  v.W1 = w;
  v.b1 = v.W1 + KO_H * KO_IN;
  v.W2 = v.b1 + KO_H;
  v.b2 = v.W2 + KO_H * KO_H;
  v.W3 = v.b2 + KO_H;
  v.b3 = v.W3 + KO_OUT * KO_H;
  return v;
}

/* One sample: a1 = W1 x + b1, h1 = relu(a1), a2 = W2 h1 + b2, h2 = relu(a2),
 * z = W3 h2 + b3.  Hidden pre-activations are returned for the backward. */
static void ko_mlp_fwd1(const ko_mlp_view* v, const double* x, double* a1, double* h1, double* a2, double* h2,
                        double* z) {
  for (int i = 0; i < KO_H; ++i) {
    double acc = v->b1[i];
    for (int k = 0; k < KO_IN; ++k) acc += v->W1[i * KO_IN + k] * x[k];
    a1[i] = acc;
    h1[i] = acc > 0.0 ? acc : 0.0;
  }
  for (int i = 0; i < KO_H; ++i) {
    double acc = v->b2[i];
    for (int k = 0; k < KO_H; ++k) acc += v->W2[i * KO_H + k] * h1[k];
    a2[i] = acc;
    h2[i] = acc > 0.0 ? acc : 0.0;
  }
  for (int i = 0; i < KO_OUT; ++i) {
    double acc = v->b3[i];
    for (int k = 0; k < KO_H; ++k) acc += v->W3[i * KO_H + k] * h2[k];
    z[i] = acc;
  }
}

/* Logits of n samples: X [n][32] -> Z [n][37]. */
int ko_mlp_forward(const double* w, const double* X, int64_t n, double* Z) {
  ko_mlp_view v = ko_mlp_split(w);
  double a1[KO_H], h1[KO_H], a2[KO_H], h2[KO_H];
  for (int64_t r = 0; r < n; ++r) ko_mlp_fwd1(&v, X + r * KO_IN, a1, h1, a2, h2, Z + r * KO_OUT);
  return 0;
}

/* Behaviour-cloning loss of n samples and its gradient.  Labels per sample:
 * side in {0 buy, 1 sell, 2 pass}, offset index in [0, 33) (tick offset + 16),
 * target log-quantity.  loss = mean over samples of
 *   -log softmax(z[0:3])[side] - log softmax(z[3:36])[offset] + (z[36] - logq)^2.
 * grad (length ko_mlp_nparam) receives d loss / d w. */
int ko_mlp_loss_grad(const double* w, const double* X, const int32_t* side, const int32_t* offset,
                     const double* logq, int64_t n, double* loss, double* grad) {
  if (n <= 0) return -1;
  ko_mlp_view v = ko_mlp_split(w);
  for (int i = 0; i < KO_NPARAM; ++i) grad[i] = 0.0;
  double* gW1 = grad;
  double* gb1 = gW1 + KO_H * KO_IN;
  double* gW2 = gb1 + KO_H;
  double* gb2 = gW2 + KO_H * KO_H;
  double* gW3 = gb2 + KO_H;
  double* gb3 = gW3 + KO_OUT * KO_H;
  double a1[KO_H], h1[KO_H], a2[KO_H], h2[KO_H], z[KO_OUT], dz[KO_OUT], dh2[KO_H], dh1[KO_H];
  double total = 0.0;
  const double inv_n = 1.0 / (double)n;
  for (int64_t r = 0; r < n; ++r) {
    const double* x = X + r * KO_IN;
    ko_mlp_fwd1(&v, x, a1, h1, a2, h2, z);
    /* softmax cross-entropy on the side head */
    double mx = z[0];
    for (int i = 1; i < KO_NSIDE; ++i) mx = z[i] > mx ? z[i] : mx;
    double se = 0.0;
    for (int i = 0; i < KO_NSIDE; ++i) se += exp(z[i] - mx);
    total += -(z[side[r]] - mx - log(se));
    for (int i = 0; i < KO_NSIDE; ++i) dz[i] = exp(z[i] - mx) / se - (i == side[r] ? 1.0 : 0.0);
    /* softmax cross-entropy on the offset head */
    mx = z[KO_NSIDE];
    for (int i = 1; i < KO_NOFF; ++i) mx = z[KO_NSIDE + i] > mx ? z[KO_NSIDE + i] : mx;
    se = 0.0;
    for (int i = 0; i < KO_NOFF; ++i) se += exp(z[KO_NSIDE + i] - mx);
    total += -(z[KO_NSIDE + offset[r]] - mx - log(se));
    for (int i = 0; i < KO_NOFF; ++i)
      dz[KO_NSIDE + i] = exp(z[KO_NSIDE + i] - mx) / se - (i == offset[r] ? 1.0 : 0.0);
    /* squared error on log-quantity */
    const double e = z[KO_OUT - 1] - logq[r];
    total += e * e;
    dz[KO_OUT - 1] = 2.0 * e;
    for (int i = 0; i < KO_OUT; ++i) dz[i] *= inv_n;
    /* layer 3 */
    for (int i = 0; i < KO_OUT; ++i) {
      gb3[i] += dz[i];
      for (int k = 0; k < KO_H; ++k) gW3[i * KO_H + k] += dz[i] * h2[k];
    }
    for (int k = 0; k < KO_H; ++k) {
      double acc = 0.0;
      for (int i = 0; i < KO_OUT; ++i) acc += v.W3[i * KO_H + k] * dz[i];
      dh2[k] = a2[k] > 0.0 ? acc : 0.0;
    }
    /* layer 2 */
    for (int i = 0; i < KO_H; ++i) {
      gb2[i] += dh2[i];
      for (int k = 0; k < KO_H; ++k) gW2[i * KO_H + k] += dh2[i] * h1[k];
    }
    for (int k = 0; k < KO_H; ++k) {
      double acc = 0.0;
      for (int i = 0; i < KO_H; ++i) acc += v.W2[i * KO_H + k] * dh2[i];
      dh1[k] = a1[k] > 0.0 ? acc : 0.0;
    }
    /* layer 1 */
    for (int i = 0; i < KO_H; ++i) {
      gb1[i] += dh1[i];
      for (int k = 0; k < KO_IN; ++k) gW1[i * KO_IN + k] += dh1[i] * x[k];
    }
  }
  *loss = total * inv_n;
  return 0;
}

/* One Adam step (Kingma and Ba, ICLR 2015) with bias correction, step t >= 1:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void ko_adam_step(double* w, const double* g, double* m, double* v, int32_t n, int32_t t, double lr, double b1,
                  double b2, double eps) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int32_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

/* Normalised policy input from the raw integer features of a decision:
 * raw[0..7]   last eight clearing-tick returns hist[j] - hist[j+1], newest first
 * raw[8]      the agent's inventory
 * raw[9]      the market's last executed volume V*
 * raw[10..13] resting sell quantity at ticks last+1 .. last+4
 * raw[14..17] resting buy quantity at ticks last-1 .. last-4
 * x = raw / (8, 256, 8A, 4A) per group, x[18..31] = 0. */
void ko_mlp_features(const int32_t* raw, int32_t A, double* x) {
  for (int j = 0; j < 8; ++j) x[j] = (double)raw[j] / 8.0;
  x[8] = (double)raw[8] / 256.0;
  x[9] = (double)raw[9] / (8.0 * (double)(A > 0 ? A : 1));
  for (int j = 10; j < KO_NRAW; ++j) x[j] = (double)raw[j] / (4.0 * (double)(A > 0 ? A : 1));
  for (int j = KO_NRAW; j < KO_IN; ++j) x[j] = 0.0;
}

/* Inverse-CDF draw from softmax(z[0..n)) with u = w / 2^32: the smallest i
 * whose cumulative probability exceeds u (the last index if rounding leaves
 * none). */
static int ko_sample(const double* z, int n, uint32_t w) {
  double mx = z[0];
  for (int i = 1; i < n; ++i) mx = z[i] > mx ? z[i] : mx;
  double se = 0.0;
  for (int i = 0; i < n; ++i) se += exp(z[i] - mx);
  const double u = (double)w / 4294967296.0;
  double c = 0.0;
  for (int i = 0; i < n; ++i) {
    c += exp(z[i] - mx) / se;
    if (u < c) return i;
  }
  return n - 1;
}

/* Action of the policy from logits z and the agent's stream-3 draw words:
 * side from w0, offset index from w1 (offset = index - 16 ticks toward the
 * opposite side), quantity clamp(round(exp(z[36])), 1, qmax). */
void ko_mlp_action(const double* z, const uint32_t w[4], int32_t qmax, int32_t* side, int32_t* offset_idx,
                   int32_t* qty) {
  *side = ko_sample(z, KO_NSIDE, w[0]);
  *offset_idx = ko_sample(z + KO_NSIDE, KO_NOFF, w[1]);
  double q = floor(exp(z[KO_OUT - 1]) + 0.5);
  if (!(q >= 1.0)) q = 1.0; /* also catches NaN */
  if (q > (double)qmax) q = (double)qmax;
  *qty = (int32_t)q;
}

/* ------------------------------------------------------------------------ */
/* Market simulation.                                                         */
/* ------------------------------------------------------------------------ */
enum { KO_ZI = 0, KO_MOM = 1, KO_MR = 2 };
#define KO_HIST 9

typedef struct {
  uint64_t seed;
  int32_t carry_book;        /* 0: unfilled orders discarded each step; 1: carried */
  uint32_t cancel_thresh;    /* a live order is cancelled iff draw word 0 < this    */
  int32_t mix_pct[3];        /* percent ZI / momentum / mean-reversion              */
  int32_t zi_offset;         /* ZI tick offset uniform in [-zi_offset, zi_offset]   */
  int32_t zi_qmax;           /* ZI quantity uniform in [1, zi_qmax]                 */
  int32_t mom_lookback;      /* momentum return horizon in steps (1..8)             */
  int32_t mom_offset_max;    /* momentum offset uniform in [0, mom_offset_max]      */
  int32_t mr_offset_max;     /* mean-reversion offset uniform in [0, mr_offset_max] */
  int32_t rb_qmax;           /* momentum / mean-reversion quantity in [1, rb_qmax]  */
  int32_t mlp_pct;           /* percent of agents driven by the MLP policy          */
  int32_t tie_rule;          /* 0 lowest tick, 1 min imbalance then lowest          */
} ko_params;

typedef struct {
  int32_t last;              /* last clearing tick (initially L/2)                  */
  int32_t hist[KO_HIST];     /* hist[j] = last clearing tick j steps ago            */
  int32_t fund;              /* per-market fundamental tick                         */
  int32_t trades;            /* steps with V* > 0                                   */
  int32_t last_v;            /* V* of the most recent step                          */
  int32_t pad_;
  int64_t sum_p;             /* sum of p* over trading steps                        */
  int64_t sum_v;             /* sum of V* over all steps                            */
  uint64_t hash;             /* running trace hash                                  */
} ko_market_scalars;

/* Per-agent arrays of one market (length A each). */
typedef struct {
  int32_t* qty;    /* working-order quantity, 0 = no working order */
  int32_t* side;   /* 0 buy, 1 sell */
  int32_t* tick;
  int32_t* atype;  /* KO_ZI / KO_MOM / KO_MR */
  int32_t* mlp;    /* 1 = decisions come from the MLP policy */
  int32_t* inv;
  int64_t* cash;
} ko_agents;

/* Initial state of market m: price L/2 everywhere in the history, no orders,
 * zero inventory and cash.  Agent class from stream 1 word 0 as a percentile;
 * MLP membership from stream 1 word 1; fundamental uniform on [L/4, 3L/4]
 * from stream 2 word 0. */
int ko_init_market(const ko_params* P, uint32_t m, int32_t L, int32_t A,
                   ko_agents* ag, ko_market_scalars* ms) {
  if (L < 2 || A < 0) return -1;
  memset(ms, 0, sizeof(*ms));
  ms->last = L / 2;
  for (int j = 0; j < KO_HIST; ++j) ms->hist[j] = L / 2;
  uint32_t w[4];
  ko_draw(P->seed, 0u, 0u, m, 2u, w);
  ms->fund = L / 4 + (int32_t)ko_range(w[0], L / 2 + 1);
  for (int32_t a = 0; a < A; ++a) {
    ko_draw(P->seed, 0u, (uint32_t)a, m, 1u, w);
    int64_t pct = ko_range(w[0], 100);
    if (pct < P->mix_pct[0]) ag->atype[a] = KO_ZI;
    else if (pct < P->mix_pct[0] + P->mix_pct[1]) ag->atype[a] = KO_MOM;
    else ag->atype[a] = KO_MR;
    ag->mlp[a] = ko_range(w[1], 100) < P->mlp_pct ? 1 : 0;
    ag->qty[a] = 0;
    ag->side[a] = 0;
    ag->tick[a] = 0;
    ag->inv[a] = 0;
    ag->cash[a] = 0;
  }
  return 0;
}

/* Rule-based decision of one agent with an empty working order, from the
 * per-step draw words w[1] (side), w[2] (offset), w[3] (quantity). */
static void ko_decide_rule(const ko_params* P, int32_t L, int32_t atype,
                           const ko_market_scalars* ms, const uint32_t w[4],
                           int32_t* side, int32_t* tick, int32_t* qty) {
  int32_t coin = (w[1] >> 31) ? 1 : 0; /* buy iff w1 < 2^31 */
  int32_t last = ms->last;
  if (atype == KO_ZI) {
    int64_t off = ko_range(w[2], 2 * (int64_t)P->zi_offset + 1) - P->zi_offset;
    *side = coin;
    *tick = ko_clamp((int64_t)last + off, 0, L - 1);
    *qty = 1 + (int32_t)ko_range(w[3], P->zi_qmax);
    return;
  }
  int32_t s;
  int64_t off;
  if (atype == KO_MOM) {
    int32_t ret = ms->hist[0] - ms->hist[P->mom_lookback];
    s = ret > 0 ? 0 : (ret < 0 ? 1 : coin);
    off = ko_range(w[2], (int64_t)P->mom_offset_max + 1);
  } else {
    s = last < ms->fund ? 0 : (last > ms->fund ? 1 : coin);
    off = ko_range(w[2], (int64_t)P->mr_offset_max + 1);
  }
  *side = s;
  *tick = ko_clamp((int64_t)last + (s == 0 ? off : -off), 0, L - 1);
  *qty = 1 + (int32_t)ko_range(w[3], P->rb_qmax);
}

/* The rule decision of an agent of class atype from its draw words w in a
 * market with scalars ms (test entry point): out = (side, tick, qty). */
void ko_rule_decision(const ko_params* P, int32_t L, int32_t atype, const ko_market_scalars* ms, const uint32_t w[4],
                      int32_t* out) {
  ko_decide_rule(P, L, atype, ms, w, &out[0], &out[1], &out[2]);
}

/* Optional replay of externally supplied decisions for MLP agents (used to
 * re-run the clearing on orders emitted by another engine).  For step j of
 * the call and agent a, entry j*A + a holds side (0 buy, 1 sell, 2 pass),
 * tick and qty; only entries of MLP agents with an empty order are read. */
typedef struct {
  const int32_t* side;
  const int32_t* tick;
  const int32_t* qty;
} ko_replay;

/* Further options of a run (all fields may be zero / NULL).
 *  mlp_w:      fp64 policy parameters; MLP agents decide with them unless a
 *              replay is given, in which case the replayed decisions are also
 *              compared with the policy's (mlp_checked / mlp_mismatch);
 *  rec_agents: rule decisions of agents a < rec_agents are recorded as
 *              KO_REC_WORDS int32 each: raw features (KO_NRAW), side,
 *              offset index, qty, agent class.  The offset counts toward
 *              the opposite side (tick - last for a buy, last - tick for a
 *              sell), clamped to [-16, 16], plus 16;
 *  logit_out:  with mlp_w, the fp64 logits of every policy decision, entry
 *              (j * A + a) * KO_OUT for step j of the call and agent a
 *              (entries without a decision are not written). */
#define KO_REC_WORDS (KO_NRAW + 4)
typedef struct {
  const double* mlp_w;
  int32_t rec_agents;
  int32_t pad_;
  int32_t* rec_out;
  int64_t rec_cap;
  int64_t rec_count;
  int64_t mlp_checked;
  int64_t mlp_mismatch;
  double* logit_out;
} ko_options;

/* Market-level raw features at the start of a step (see ko_mlp_features). */
static void ko_raw_features(const ko_market_scalars* ms, int32_t L, const int64_t* buy, const int64_t* sell,
                            int32_t* raw) {
  for (int j = 0; j < 8; ++j) raw[j] = ms->hist[j] - ms->hist[j + 1];
  raw[8] = 0;
  raw[9] = ms->last_v;
  for (int k = 1; k <= 4; ++k) {
    int32_t pa = ms->last + k, pb = ms->last - k;
    raw[9 + k] = (pa >= 0 && pa < L) ? (int32_t)sell[pa] : 0;
    raw[13 + k] = (pb >= 0 && pb < L) ? (int32_t)buy[pb] : 0;
  }
}

/* The policy's decision for agent a at step s (fp64); z_out (nullable)
 * receives its logits. */
static void ko_mlp_decide(const ko_params* P, const double* w, uint32_t m, int32_t L, int32_t A, uint32_t s,
                          int32_t a, const int32_t* raw_mkt, int32_t inv, int32_t last, int32_t* side,
                          int32_t* tick, int32_t* qty, double* z_out) {
  int32_t raw[KO_NRAW];
  memcpy(raw, raw_mkt, sizeof(raw));
  raw[8] = inv;
  double x[KO_IN], z[KO_OUT];
  ko_mlp_features(raw, A, x);
  ko_mlp_forward(w, x, 1, z);
  if (z_out) memcpy(z_out, z, sizeof(z));
  uint32_t u[4];
  ko_draw(P->seed, s, (uint32_t)a, m, 3u, u);
  int32_t oi;
  ko_mlp_action(z, u, P->rb_qmax, side, &oi, qty);
  /* the offset counts toward the opposite side: up for a buy, down for a sell */
  const int32_t k = oi - KO_OFF_MAX;
  *tick = ko_clamp((int64_t)last + (*side == 1 ? -k : k), 0, L - 1);
}

/* Run steps [s0, s0 + n) of market m.  trace_p / trace_v (nullable, length n)
 * receive p* (-1 for no trade) and V* per step.  Returns 0 on success. */
int ko_run_market(const ko_params* P, uint32_t m, int32_t L, int32_t A, ko_agents* ag,
                  ko_market_scalars* ms, uint32_t s0, uint32_t n, const ko_replay* replay,
                  int32_t* trace_p, int32_t* trace_v, ko_options* opt) {
  if (L < 2 || A < 0) return -1;
  int64_t* buy = (int64_t*)calloc((size_t)L, sizeof(int64_t));
  int64_t* sell = (int64_t*)calloc((size_t)L, sizeof(int64_t));
  int64_t* dcum = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
  int64_t* scum = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
  int64_t* vol = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
  int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A > 0 ? A : 1));
  int rc = 0;
  int any_mlp = 0;
  for (int32_t a = 0; a < A; ++a) any_mlp |= ag->mlp[a];
  const double* mlp_w = opt ? opt->mlp_w : NULL;
  const int32_t rec_agents = opt ? opt->rec_agents : 0;
  if (!buy || !sell || !dcum || !scum || !vol || !fill) { rc = -2; goto done; }
  for (uint32_t j = 0; j < n; ++j) {
    uint32_t s = s0 + j;
    /* resting book at the start of the step: the inputs of the policy features */
    int32_t raw_mkt[KO_NRAW];
    if (any_mlp || rec_agents > 0) {
      for (int32_t p = 0; p < L; ++p) { buy[p] = 0; sell[p] = 0; }
      for (int32_t a = 0; a < A; ++a) {
        if (ag->qty[a] <= 0) continue;
        if (ag->side[a] == 0) buy[ag->tick[a]] += ag->qty[a];
        else sell[ag->tick[a]] += ag->qty[a];
      }
      ko_raw_features(ms, L, buy, sell, raw_mkt);
    }
    /* 1-2. cancellation of working orders, then decisions of empty agents */
    for (int32_t a = 0; a < A; ++a) {
      uint32_t w[4];
      ko_draw(P->seed, s, (uint32_t)a, m, 0u, w);
      if (P->carry_book && ag->qty[a] > 0 && w[0] < P->cancel_thresh) ag->qty[a] = 0;
      if (ag->qty[a] > 0) continue;
      if (ag->mlp[a]) {
        int32_t sd, tk, q;
        if (replay) {
          size_t e = (size_t)j * (size_t)A + (size_t)a;
          sd = replay->side[e];
          tk = replay->tick[e];
          q = replay->qty[e];
          if (sd < 0 || sd > 2 || (sd < 2 && (tk < 0 || tk >= L || q <= 0))) { rc = -6; goto done; }
          if (mlp_w) {
            int32_t os, ot, oq;
            ko_mlp_decide(P, mlp_w, m, L, A, s, a, raw_mkt, ag->inv[a], ms->last, &os, &ot, &oq,
                          opt->logit_out ? opt->logit_out + ((size_t)j * (size_t)A + (size_t)a) * KO_OUT : NULL);
            opt->mlp_checked += 1;
            if (os != sd || (sd < 2 && (ot != tk || oq != q))) opt->mlp_mismatch += 1;
          }
        } else {
          if (!mlp_w) { rc = -5; goto done; }
          ko_mlp_decide(P, mlp_w, m, L, A, s, a, raw_mkt, ag->inv[a], ms->last, &sd, &tk, &q,
                        opt->logit_out ? opt->logit_out + ((size_t)j * (size_t)A + (size_t)a) * KO_OUT : NULL);
        }
        if (sd == 2) continue; /* pass: no order this step */
        ag->side[a] = sd;
        ag->tick[a] = tk;
        ag->qty[a] = q;
        continue;
      }
      ko_decide_rule(P, L, ag->atype[a], ms, w, &ag->side[a], &ag->tick[a], &ag->qty[a]);
      if (a < rec_agents && opt->rec_out && opt->rec_count < opt->rec_cap) {
        int32_t* r = opt->rec_out + opt->rec_count * KO_REC_WORDS;
        memcpy(r, raw_mkt, sizeof(raw_mkt));
        r[8] = ag->inv[a];
        int32_t off = ag->side[a] == 1 ? ms->last - ag->tick[a] : ag->tick[a] - ms->last;
        off = off < -KO_OFF_MAX ? -KO_OFF_MAX : (off > KO_OFF_MAX ? KO_OFF_MAX : off);
        r[KO_NRAW + 0] = ag->side[a];
        r[KO_NRAW + 1] = off + KO_OFF_MAX;
        r[KO_NRAW + 2] = ag->qty[a];
        r[KO_NRAW + 3] = ag->atype[a];
        opt->rec_count += 1;
      }
    }
    /* 3. aggregated book of all working orders */
    for (int32_t p = 0; p < L; ++p) { buy[p] = 0; sell[p] = 0; }
    for (int32_t a = 0; a < A; ++a) {
      if (ag->qty[a] <= 0) continue;
      if (ag->side[a] == 0) buy[ag->tick[a]] += ag->qty[a];
      else sell[ag->tick[a]] += ag->qty[a];
    }
    /* 4. clearing */
    ko_clear_result cr;
    if (ko_clear_book(L, buy, sell, P->tie_rule, dcum, scum, vol, &cr) != 0) { rc = -3; goto done; }
    if (dcum[0] > INT32_MAX || scum[L - 1] > INT32_MAX) { rc = -7; goto done; }
    /* 5. allocation and accounts at the single price p* */
    if (cr.vstar > 0) {
      int r = ko_allocate(L, A, ag->side, ag->tick, ag->qty, cr.vstar, fill);
      if (r != 0) { rc = -4; goto done; }
      for (int32_t a = 0; a < A; ++a) {
        int32_t f = fill[a];
        if (f == 0) continue;
        if (ag->side[a] == 0) {
          ag->inv[a] += f;
          ag->cash[a] -= (int64_t)cr.pstar * f;
        } else {
          ag->inv[a] -= f;
          ag->cash[a] += (int64_t)cr.pstar * f;
        }
        ag->qty[a] -= f;
      }
      ms->last = cr.pstar;
      ms->sum_p += cr.pstar;
      ms->sum_v += cr.vstar;
      ms->trades += 1;
    }
    /* 6. discard mode: no order survives the step */
    if (!P->carry_book)
      for (int32_t a = 0; a < A; ++a) ag->qty[a] = 0;
    /* 7. price history, statistics and trace hash */
    for (int k = KO_HIST - 1; k > 0; --k) ms->hist[k] = ms->hist[k - 1];
    ms->hist[0] = ms->last;
    ms->last_v = (int32_t)cr.vstar;
    ms->hash = ko_trace_hash_update(ms->hash, s, cr.pstar, (int32_t)cr.vstar);
    if (trace_p) trace_p[j] = cr.pstar;
    if (trace_v) trace_v[j] = (int32_t)cr.vstar;
  }
done:
  free(buy); free(sell); free(dcum); free(scum); free(vol); free(fill);
  return rc;
}

/* ======================================================================== */
/* The paper's own agents (Sec. III-C, "Agent Decision and Order            */
/* Aggregation") on a tick-aggregated book with SplitMix64 draws (Sec.      */
/* III-G).  Readings where the paper is silent (each marked READING):        */
/*  - draws: u(gid, s, c) = mix64(seed + 0x9E3779B97F4A7C15 * (gid * 2^35 +   */
/*    8 s + c)) mod 2^64, i.e. output number gid*2^35 + 8s + c of the         */
/*    SplitMix64 generator with state `seed` (Steele, Lea, Flood, OOPSLA      */
/*    2014); gid = market * A + a is the paper's global agent id.  Channel 0: */
/*    high word = marketable draw, low word = side coin (bit 31); channel 1:  */
/*    high word = price draw, low word = quantity draw; channel 2 at step 0:  */
/*    high word = agent class draw.                                          */
/*  - class: percentile floor(100 w / 2^32) of the class draw; MAKER below    */
/*    maker_pct, MOMENTUM below maker_pct + mom_pct, NOISE otherwise.         */
/*  - the clearing takes the step's own orders (Algorithm 1 scans s_BUY and   */
/*    s_SELL); their unfilled part (the worked example's new_bid = BUY -      */
/*    traded_buy) replaces the resting book, which feeds the next step's mid. */
/*  - round(x) = the nearest integer, ties to even (IEEE-754 round to        */
/*    nearest); a round-half-up rule shifts both maker quotes up by half a    */
/*    tick whenever the spread is odd, a ratchet that walks the price to the  */
/*    top of the grid.  Ticks are clamped to [0, L).                           */
/*  - the first step's previous mid is the opening mid L/2 (integer part).   */
/*  - sliding window (Sec. III-A: the grid is a local window of L ticks      */
/*    around the trading zone; the recentring rule is not given).  With      */
/*    `window` set, absolute tick = base + window tick.  At the start of a    */
/*    step, after the mid is found, the window moves when the mid is more    */
/*    than L/4 from its centre c = L/2: by k = 2 floor((2 mid - 2c) / 4)     */
/*    ticks, an even number, so that ties-to-even rounding in the window is  */
/*    the same rounding in absolute ticks.  The mid and the last price move  */
/*    with it (the sign of the mid change is taken before the move); the     */
/*    resting book is not moved because the step's own orders replace it.    */
/*    Orders beyond the window are clamped to its edge                       */
/*    (executed as marketable); marketable orders go to the window's edges.  */
/*    Traces then record the absolute last price after each step (carried   */
/*    on steps without trade) and V*; Sum p* and the hash take absolute p*.  */
/* ======================================================================== */
#define KO_PAPER_NOISE 0
#define KO_PAPER_MOMENTUM 1
#define KO_PAPER_MAKER 2

typedef struct {
  uint64_t seed;
  int32_t noise_halfwidth;   /* Delta_noise, ticks                            */
  uint32_t p_mkt_q32;        /* P_mkt * 2^32                                  */
  int32_t qmax;              /* q_max                                         */
  int32_t maker_half_spread; /* Delta_maker_half_spread, ticks                */
  int32_t mom_pct;           /* alpha_mom in percent                          */
  int32_t maker_pct;         /* alpha_maker in percent                        */
  int32_t tie_rule;
  int32_t window;            /* 1: sliding window with recentring            */
} ko_paper_params;

typedef struct {
  int32_t last;    /* last clearing tick                                      */
  int32_t mid2;    /* twice the mid of the latest step (the next step's mid_{t-1}) */
  int32_t trades;
  int32_t last_v;
  int64_t sum_p;
  int64_t sum_v;
  uint64_t hash;
  int64_t base;    /* absolute tick of window tick 0 (0 without a window)    */
} ko_paper_market;

/* floor(num / den) for den > 0 */
static int64_t ko_floor_div(int64_t num, int64_t den) {
  int64_t q = num / den;
  if ((num % den) != 0 && num < 0) q -= 1;
  return q;
}

/* num / den rounded to the nearest integer, ties to even (den > 0, even) */
static int64_t ko_round_even(int64_t num, int64_t den) {
  int64_t q = ko_floor_div(num, den);
  int64_t r = num - q * den;      /* 0 <= r < den */
  if (2 * r > den) return q + 1;
  if (2 * r < den) return q;
  return (q % 2 != 0) ? q + 1 : q;
}

uint64_t ko_splitmix64_draw(uint64_t seed, uint64_t gid, uint32_t step, uint32_t channel) {
  uint64_t counter = gid * (1ull << 35) + (uint64_t)step * 8ull + (uint64_t)channel;
  return ko_mix64(seed + 0x9E3779B97F4A7C15ull * counter);
}

int32_t ko_paper_class(const ko_paper_params* P, uint64_t gid) {
  uint32_t w = (uint32_t)(ko_splitmix64_draw(P->seed, gid, 0, 2) >> 32);
  int64_t pct = ko_range(w, 100);
  if (pct < P->maker_pct) return KO_PAPER_MAKER;
  if (pct < P->maker_pct + P->mom_pct) return KO_PAPER_MOMENTUM;
  return KO_PAPER_NOISE;
}

/* Order of agent a (class cls) at step s given the step's mid (mid2 = 2 mid)
 * and the sign of the mid change ret: side 0 buy / 1 sell, tick, qty. */
void ko_paper_order(const ko_paper_params* P, int32_t L, uint64_t gid, int32_t a, uint32_t s, int32_t cls,
                    int32_t mid2, int32_t ret, int32_t* side, int32_t* tick, int32_t* qty) {
  uint64_t u0 = ko_splitmix64_draw(P->seed, gid, s, 0);
  uint64_t u1 = ko_splitmix64_draw(P->seed, gid, s, 1);
  uint32_t w_mkt = (uint32_t)(u0 >> 32), w_coin = (uint32_t)u0;
  uint32_t w_price = (uint32_t)(u1 >> 32), w_qty = (uint32_t)u1;
  int32_t sd;
  int64_t p;
  if (cls == KO_PAPER_MAKER) {
    /* buys iff (a + s) mod 2 = 0; bid at round(mid - D), ask at round(mid + D) */
    sd = (int32_t)(((int64_t)a + (int64_t)s) % 2);
    int64_t D = P->maker_half_spread;
    p = ko_round_even((int64_t)mid2 + (sd ? 2 * D : -2 * D), 2);
  } else {
    if (cls == KO_PAPER_MOMENTUM && ret != 0)
      sd = ret > 0 ? 0 : 1;                 /* side = sign of the mid change */
    else
      sd = (w_coin >= 0x80000000u) ? 1 : 0; /* buy or sell with equal probability */
    if (w_mkt < P->p_mkt_q32) {
      p = sd ? 0 : L - 1;                   /* marketable: the grid boundary */
    } else if (cls == KO_PAPER_MOMENTUM) {
      p = ko_round_even((int64_t)mid2 + (sd ? -2 : 2), 2);   /* round(mid + side) */
    } else {
      /* round(mid + eta), eta = -D + 2 D w / 2^32: numerator over 2^33 */
      int64_t D = P->noise_halfwidth;
      int64_t num = ((int64_t)mid2 - 2 * D) * (1ll << 32) + 4 * D * (int64_t)w_price;
      p = ko_round_even(num, 1ll << 33);
    }
  }
  *side = sd;
  *tick = ko_clamp(p, 0, L - 1);
  *qty = (int32_t)(1 + ko_range(w_qty, P->qmax));
}

int ko_paper_init(int32_t L, int32_t* bid, int32_t* ask, ko_paper_market* ms) {
  if (L < 2) return -1;
  for (int32_t p = 0; p < L; ++p) bid[p] = ask[p] = 0;
  memset(ms, 0, sizeof(*ms));
  ms->last = L / 2;
  ms->mid2 = 2 * (L / 2);
  return 0;
}

/* Steps [s0, s0 + n) of global market `market`; trace: 2 int32 per step or NULL. */
int ko_paper_run(const ko_paper_params* P, uint32_t market, int32_t L, int32_t A, int32_t* bid, int32_t* ask,
                 ko_paper_market* ms, uint32_t s0, uint32_t n, int32_t* trace) {
  if (L < 2 || A < 0) return -1;
  int64_t* buy = (int64_t*)calloc((size_t)L, sizeof(int64_t));
  int64_t* sell = (int64_t*)calloc((size_t)L, sizeof(int64_t));
  int64_t* dcum = (int64_t*)calloc((size_t)L, sizeof(int64_t));
  int64_t* scum = (int64_t*)calloc((size_t)L, sizeof(int64_t));
  int64_t* vol = (int64_t*)calloc((size_t)L, sizeof(int64_t));
  int32_t* cls = (int32_t*)calloc((size_t)(A > 0 ? A : 1), sizeof(int32_t));
  int rc = 0;
  if (!buy || !sell || !dcum || !scum || !vol || !cls) { rc = -2; goto done; }
  for (int32_t a = 0; a < A; ++a) cls[a] = ko_paper_class(P, (uint64_t)market * (uint64_t)A + (uint64_t)a);
  for (uint32_t j = 0; j < n; ++j) {
    uint32_t s = s0 + j;
    /* state retrieval: best bid / ask of the resting book, mid price */
    int32_t bb = -1, ba = L;
    for (int32_t p = 0; p < L; ++p)
      if (bid[p] > 0) bb = p;
    for (int32_t p = L - 1; p >= 0; --p)
      if (ask[p] > 0) ba = p;
    int32_t mid2 = (bb >= 0 && ba < L) ? bb + ba : 2 * ms->last;
    int32_t ret = (mid2 > ms->mid2) - (mid2 < ms->mid2);
    if (P->window) {
      /* recentre when |mid - L/2| > L/4 (in half ticks: |mid2 - c2| > L/2) */
      int32_t dev = mid2 - 2 * (L / 2);
      if (dev > L / 2 || dev < -(L / 2)) {
        int32_t k = 2 * (int32_t)ko_floor_div(dev, 4);
        ms->base += k;
        mid2 -= 2 * k;
        ms->last -= k;
      }
    }
    /* the step's orders */
    for (int32_t p = 0; p < L; ++p) buy[p] = sell[p] = 0;
    for (int32_t a = 0; a < A; ++a) {
      int32_t sd, tk, q;
      ko_paper_order(P, L, (uint64_t)market * (uint64_t)A + (uint64_t)a, a, s, cls[a], mid2, ret, &sd, &tk, &q);
      if (sd) sell[tk] += q; else buy[tk] += q;
    }
    /* clearing */
    ko_clear_result cr;
    ko_clear_book(L, buy, sell, P->tie_rule, dcum, scum, vol, &cr);
    /* the unfilled part of the step's orders becomes the resting book */
    for (int32_t p = 0; p < L; ++p) {
      int64_t nb = buy[p], na = sell[p];
      if (cr.vstar > 0) {
        int64_t above_b = p + 1 < L ? dcum[p + 1] : 0;  /* demand strictly above p */
        int64_t below_s = p > 0 ? scum[p - 1] : 0;      /* supply strictly below p */
        if (p > cr.p_buy) nb = 0;
        else if (p == cr.p_buy) nb = buy[p] - (cr.vstar - above_b);
        if (p < cr.p_sell) na = 0;
        else if (p == cr.p_sell) na = sell[p] - (cr.vstar - below_s);
      }
      if (nb > 0x7FFFFFFF || na > 0x7FFFFFFF) { rc = -3; goto done; }
      bid[p] = (int32_t)nb;
      ask[p] = (int32_t)na;
    }
    if (cr.vstar > 0x7FFFFFFF) { rc = -3; goto done; }
    int32_t pabs = cr.vstar > 0 ? (int32_t)(ms->base + cr.pstar) : -1;  /* absolute p*, -1 without trade */
    if (cr.vstar > 0) {
      ms->last = cr.pstar;
      ms->trades += 1;
      ms->sum_p += ms->base + cr.pstar;
    }
    ms->sum_v += cr.vstar;
    ms->last_v = (int32_t)cr.vstar;
    ms->mid2 = mid2;
    ms->hash = ko_trace_hash_update(ms->hash, s, pabs, (int32_t)cr.vstar);
    if (trace) {
      trace[2 * j] = P->window ? (int32_t)(ms->base + ms->last) : pabs;
      trace[2 * j + 1] = (int32_t)cr.vstar;
    }
  }
done:
  free(buy); free(sell); free(dcum); free(scum); free(vol); free(cls);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Continuous double auction (the pattern's generalisation the paper names    */
/* in its discussion section; its rules are readings C1-C6).                  */
/*                                                                            */
/* The agents, draws, cancellation and rule decisions are the main model's.   */
/* Each step: C1 every working order is cancelled with its step-s draw;       */
/* C2 every agent without a working order decides from the step-start state  */
/* (the rule of ko_decide_rule); C3 the new orders arrive one by one in       */
/* ascending agent index and each trades at once against the opposite side   */
/* in price-time priority: the best price first, at a price the earliest     */
/* arrival first, each fill at the resting order's tick, while the incoming  */
/* limit still crosses; the remainder rests with arrival stamp s * A + a.    */
/* C4 every fill moves inventory and cash at the fill's tick.  C5 the step's  */
/* last clearing tick is that of its last fill (unchanged without fills), the */
/* history shifts it in, trades counts fills, sum_p adds tick * qty of every  */
/* fill, sum_v and last_v the step's volume, and the trace hash folds (last   */
/* fill tick or -1, step volume).  C6 the resting book has no identity beyond */
/* (side, tick, stamp): it is plain per-agent state, and price-time priority  */
/* is evaluated by scanning the agents (slow and plain).                      */
/* ------------------------------------------------------------------------ */

/* The resting order that an incoming order of side `side` (0 buy, 1 sell)
 * with limit `tick` trades against next: the best opposite price that
 * crosses, among those the smallest stamp; -1 if none crosses. */
static int32_t ko_cda_best(int32_t A, const ko_agents* ag, const int64_t* stamp, int32_t side, int32_t tick) {
  int32_t best = -1;
  for (int32_t b = 0; b < A; ++b) {
    if (ag->qty[b] <= 0 || ag->side[b] == side) continue;
    const int32_t t = ag->tick[b];
    if (side == 0 ? t > tick : t < tick) continue; /* does not cross the limit */
    if (best < 0) { best = b; continue; }
    const int32_t tb = ag->tick[best];
    const int better = side == 0 ? (t < tb) : (t > tb);
    if (better || (t == tb && stamp[b] < stamp[best])) best = b;
  }
  return best;
}

/* Run steps [s0, s0 + n) of CDA market m.  stamp[a]: arrival stamp of a's
 * resting order (-1 if none).  trace_p / trace_v (nullable) receive the last
 * fill tick (-1 without fills) and the volume of each step.  fills (nullable,
 * fills_cap rows of 5 int32: step, incoming agent, resting agent, tick, qty)
 * receives the fill log, *fills_count the number of fills (also beyond the
 * capacity).  inject (nullable, test use): entry j * A + a replaces the
 * decision of agent a at step j of the call if it decides (qty <= 0: no
 * order).  Returns 0 on success. */
int ko_cda_run(const ko_params* P, uint32_t m, int32_t L, int32_t A, ko_agents* ag, int64_t* stamp,
               ko_market_scalars* ms, uint32_t s0, uint32_t n, int32_t* trace_p, int32_t* trace_v, int32_t* fills,
               int64_t fills_cap, int64_t* fills_count, const ko_replay* inject) {
  if (L < 2 || A < 0) return -1;
  for (int32_t a = 0; a < A; ++a)
    if (ag->mlp[a]) return -5; /* policy agents are not part of this model */
  int32_t* dside = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A > 0 ? A : 1));
  int32_t* dtick = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A > 0 ? A : 1));
  int32_t* dqty = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A > 0 ? A : 1));
  if (!dside || !dtick || !dqty) { free(dside); free(dtick); free(dqty); return -2; }
  int64_t nf = fills_count ? *fills_count : 0;
  for (uint32_t j = 0; j < n; ++j) {
    const uint32_t s = s0 + j;
    /* C1 cancellations and C2 decisions, all from the step-start state */
    for (int32_t a = 0; a < A; ++a) {
      uint32_t w[4];
      ko_draw(P->seed, s, (uint32_t)a, m, 0u, w);
      dqty[a] = 0;
      if (ag->qty[a] > 0 && w[0] < P->cancel_thresh) {
        ag->qty[a] = 0;
        stamp[a] = -1;
      }
      if (ag->qty[a] > 0) continue;
      if (inject) {
        const size_t e = (size_t)j * (size_t)A + (size_t)a;
        dside[a] = inject->side[e];
        dtick[a] = inject->tick[e];
        dqty[a] = inject->qty[e];
        if (dqty[a] > 0 && (dside[a] < 0 || dside[a] > 1 || dtick[a] < 0 || dtick[a] >= L)) {
          free(dside); free(dtick); free(dqty);
          return -6;
        }
        continue;
      }
      ko_decide_rule(P, L, ag->atype[a], ms, w, &dside[a], &dtick[a], &dqty[a]);
    }
    /* C3 arrivals in agent order */
    int64_t vol = 0;
    int32_t last_fill = -1;
    for (int32_t a = 0; a < A; ++a) {
      int32_t q = dqty[a];
      if (q <= 0) continue;
      const int32_t sd = dside[a], tk = dtick[a];
      while (q > 0) {
        const int32_t r = ko_cda_best(A, ag, stamp, sd, tk);
        if (r < 0) break;
        const int32_t px = ag->tick[r];
        const int32_t f = q < ag->qty[r] ? q : ag->qty[r];
        /* C4 accounts at the resting order's tick */
        if (sd == 0) {
          ag->inv[a] += f; ag->cash[a] -= (int64_t)px * f;
          ag->inv[r] -= f; ag->cash[r] += (int64_t)px * f;
        } else {
          ag->inv[a] -= f; ag->cash[a] += (int64_t)px * f;
          ag->inv[r] += f; ag->cash[r] -= (int64_t)px * f;
        }
        ag->qty[r] -= f;
        if (ag->qty[r] == 0) stamp[r] = -1;
        q -= f;
        vol += f;
        last_fill = px;
        ms->trades += 1;
        ms->sum_p += (int64_t)px * f;
        if (fills && nf < fills_cap) {
          int32_t* e = fills + 5 * nf;
          e[0] = (int32_t)s; e[1] = a; e[2] = r; e[3] = px; e[4] = f;
        }
        nf += 1;
      }
      if (q > 0) { /* the remainder rests */
        ag->side[a] = sd;
        ag->tick[a] = tk;
        ag->qty[a] = q;
        stamp[a] = (int64_t)s * (int64_t)A + a;
      }
    }
    /* C5 step statistics */
    if (vol > 0x7FFFFFFF) { free(dside); free(dtick); free(dqty); return -7; }
    if (last_fill >= 0) ms->last = last_fill;
    for (int k = KO_HIST - 1; k > 0; --k) ms->hist[k] = ms->hist[k - 1];
    ms->hist[0] = ms->last;
    ms->last_v = (int32_t)vol;
    ms->sum_v += vol;
    ms->hash = ko_trace_hash_update(ms->hash, s, last_fill, (int32_t)vol);
    if (trace_p) trace_p[j] = last_fill;
    if (trace_v) trace_v[j] = (int32_t)vol;
  }
  if (fills_count) *fills_count = nf;
  free(dside); free(dtick); free(dqty);
  return 0;
}
