/*
 * kineticsim.h -- C ABI of the GB300 persistent call-auction engine.
 *
 * One ensemble = M independent limit-order-book markets, each with L integer
 * price ticks and A agents, advanced S steps at a time by one persistent
 * sm_103a kernel that keeps each market's book and agent orders on chip for
 * all steps of a call (the paper's Algorithm 1: inputs M markets, S steps,
 * A agents, L price levels; output the final book and clearing statistics in
 * global memory).
 *
 * Every step of every market:
 *   1. each working order is cancelled with a fixed probability (carried
 *      books only), then every agent without a working order draws a new
 *      limit order (side, tick, qty) from one Philox4x32-10 block keyed by
 *      (seed, market, agent, step);
 *   2. orders are aggregated into per-tick BUY / SELL quantities;
 *   3. D_cum[p] = sum_{q>=p} BUY[q], S_cum[p] = sum_{q<=p} SELL[q]
 *      (Sec. II-A, Eq. 1), the clearing tick p* maximises
 *      V(p) = min(D_cum[p], S_cum[p]) with ties to the lowest tick
 *      (Eq. 2, Sec. III-D);
 *   4. V* = V(p*) units trade at p*: buys fill in price priority from the top
 *      tick, sells from the bottom tick, ascending agent index within a tick
 *      (Sec. IV-C); inventory and cash of each agent are updated;
 *   5. unfilled quantity rests for the next step (carried book) or is
 *      discarded.
 * All quantities are integers; results are bit-identical for any launch
 * shape and any split of the steps over calls.
 *
 * Conventions for every function:
 *  - Returns KS_OK (0) on success.  No function throws or aborts.
 *  - Argument errors are reported before any GPU work is queued.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *  - Device memory is owned by the caller: the library never allocates
 *    device memory.  Host memory it needs (the handle) is freed by
 *    ks_destroy.
 *  - On KS_ERR_CUDA, ks_last_error() returns the CUDA error text of the
 *    calling thread's most recent failure.
 */
#ifndef KINETICSIM_H
#define KINETICSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ks_status {
  KS_OK = 0,
  KS_ERR_INVALID_ARG = 1,         /* bad pointer, size or parameter value           */
  KS_ERR_WORKSPACE_TOO_SMALL = 2, /* ws_bytes below ks_workspace_size()             */
  KS_ERR_CUDA = 3,                /* a CUDA runtime call failed (see ks_last_error) */
  KS_ERR_UNSUPPORTED = 4,         /* outside the supported envelope (L, A, qty)     */
  KS_ERR_DEVICE_FAULT = 5,        /* a kernel set the ensemble's device error word  */
  KS_ERR_TIMEOUT = 6              /* ks_sync deadline passed before the GPU finished */
} ks_status;

/* Tie rule among ticks of equal maximal executable volume. */
typedef enum ks_tie_rule {
  KS_TIE_LOWEST_TICK = 0,   /* the paper's rule (Sec. III-D): lowest price index    */
  KS_TIE_MIN_IMBALANCE = 1  /* smallest |D_cum - S_cum|, then lowest tick           */
} ks_tie_rule;

/* Supported envelope. */
#define KS_MAX_TICKS 4096   /* L in [2, 4096]                                      */
#define KS_MAX_AGENTS 16384 /* A in [1, 16384]                                     */
#define KS_MAX_QTY 255      /* zi_qmax, rb_qmax in [1, 255]                        */
#define KS_HISTORY 9        /* clearing-tick history kept per market               */

/* Agent classes (stored in the order word, see below). */
#define KS_CLASS_ZI 0   /* zero-intelligence: side 1/2, tick last +/- zi_offset      */
#define KS_CLASS_MOM 1  /* momentum: side = sign of the mom_lookback-step return    */
#define KS_CLASS_MR 2   /* mean reversion toward the market's fundamental tick      */

/*
 * Ensemble description.  Host arrays are copied by ks_create_ensemble.
 *
 * Agent rules (every draw is one word of the agent's Philox4x32-10 block for
 * counter (step, agent, market, 0) under key (seed low 32, seed high 32);
 * range(w, n) = floor(w * n / 2^32)):
 *  - cancel: a working order is cancelled iff w0 < cancel_thresh_q32;
 *  - ZI:  buy iff w1 < 2^31; tick = clamp(last + range(w2, 2*zi_offset+1)
 *         - zi_offset, 0, L-1); qty = 1 + range(w3, zi_qmax);
 *  - MOM: r = hist[0] - hist[mom_lookback]; buy if r > 0, sell if r < 0,
 *         else the ZI side bit; tick = last +/- range(w2, mom_offset_max+1)
 *         (buy above, sell below), clamped; qty = 1 + range(w3, rb_qmax);
 *  - MR:  buy if last < fundamental, sell if above, else the side bit;
 *         tick = last +/- range(w2, mr_offset_max+1); qty as MOM.
 * Here `market` is the global index market_base + m.
 * Agent class: percentile range(w0, 100) of block (0, agent, market, 1)
 * against mix_pct; MLP membership: range(w1, 100) < mlp_pct of that block.
 * Fundamental: L/4 + range(w0, L/2+1) of block (0, 0, market, 2).
 */
typedef struct ks_config {
  uint32_t n_markets;          /* M >= 1                                          */
  uint32_t market_base;        /* global index of market 0; market m draws with
                                  market word market_base + m (shards of one
                                  larger ensemble use disjoint ranges)            */
  const int32_t* L;            /* host [M] ticks per market, or NULL -> L_all      */
  const int32_t* A;            /* host [M] agents per market, or NULL -> A_all     */
  int32_t L_all;
  int32_t A_all;
  uint64_t seed;
  int32_t carry_book;          /* 0: unfilled orders discarded every step; 1: kept */
  uint32_t cancel_thresh_q32;  /* per-step cancel probability * 2^32               */
  uint32_t mix_pct[3];         /* percent ZI / MOM / MR, sum 100                   */
  int32_t zi_offset;           /* >= 0                                             */
  int32_t zi_qmax;             /* 1..KS_MAX_QTY                                    */
  int32_t mom_lookback;        /* 1..8                                             */
  int32_t mom_offset_max;      /* >= 0                                             */
  int32_t mr_offset_max;       /* >= 0                                             */
  int32_t rb_qmax;             /* 1..KS_MAX_QTY                                    */
  uint32_t mlp_pct;            /* percent of agents driven by the MLP policy       */
  const void* mlp_params;      /* device pointer to packed policy weights, or NULL */
  int32_t tie_rule;            /* ks_tie_rule                                      */
  uint32_t trace_markets;      /* markets 0..trace_markets-1 record a step trace   */
  uint32_t trace_steps;        /* trace capacity in steps (absolute steps < this)  */
} ks_config;

typedef struct ks_ensemble ks_ensemble;

/*
 * Order word (one uint32 per agent):
 *   bits 0-7   quantity of the working order (0 = no working order)
 *   bit  8     side (0 buy, 1 sell)
 *   bits 9-20  limit tick
 *   bits 21-22 agent class (KS_CLASS_*)
 *   bit  23    MLP-driven agent (an ensemble without a policy network ignores
 *              it: its agents follow their rule)
 */
#define KS_ORDER_QTY(w) ((int32_t)((w) & 0xFFu))
#define KS_ORDER_SIDE(w) ((int32_t)(((w) >> 8) & 1u))
#define KS_ORDER_TICK(w) ((int32_t)(((w) >> 9) & 0xFFFu))
#define KS_ORDER_CLASS(w) ((int32_t)(((w) >> 21) & 3u))
#define KS_ORDER_MLP(w) ((int32_t)(((w) >> 23) & 1u))

/*
 * State view: caller-owned buffers, host or device (any mix; copies use
 * unified addressing).  A NULL field is skipped.  Agent arrays are indexed by
 * the global agent id: market m's agents are [off_m, off_m + A_m) with
 * off_m = A_0 + ... + A_{m-1}; N = off_M.
 */
typedef struct ks_state_view {
  uint32_t* order;       /* [N] order words                                     */
  int32_t* inventory;    /* [N] shares bought minus sold                         */
  int64_t* cash;         /* [N] sum of p* x (sold - bought), tick units           */
  int32_t* last_tick;    /* [M] last clearing tick (initially L/2)               */
  int32_t* history;      /* [M*KS_HISTORY] history[m*9 + j] = last tick j steps ago */
  int32_t* fundamental;  /* [M]                                                 */
  int32_t* trades;       /* [M] steps with V* > 0                                */
  int32_t* last_volume;  /* [M] V* of the latest step                            */
  int64_t* sum_price;    /* [M] sum of p* over trading steps                      */
  int64_t* sum_volume;   /* [M] sum of V* over steps                             */
  uint64_t* trace_hash;  /* [M] h <- mix64(h ^ (p*<<32 | V*) ^ step*0x9E3779B97F4A7C15),
                            mix64 = SplitMix64 finaliser (Sec. III-G); p* = -1 when V* = 0 */
  uint64_t* step;        /* [1] absolute step counter                            */
  int32_t* trace;        /* [trace_markets*trace_steps*2] (p*, V*) per market and step */
} ks_state_view;

/* Launch shape of the persistent kernel; results never depend on it. */
typedef struct ks_launch {
  int32_t threads;            /* threads per CTA: 64, 128, 256, 512 or 1024      */
  int32_t agents_per_thread;  /* 1, 2, 4, 8 or 16; threads*agents_per_thread >= A */
  int32_t ctas_per_sm;        /* 0 = as many as fit                               */
  int32_t aggregate;          /* 1 = warp-aggregate equal (side,tick) orders with
                                 __match_any_sync before the shared atomic         */
  int32_t reg_cap;            /* register cap class: 0 compiler's choice, 1 at most
                                 128 registers per thread (two 256-thread CTAs per
                                 SM), 2 at most 85 (three; 128- and 256-thread CTAs
                                 with 1, 2 or 4 agents per thread, aggregate = 0),
                                 3 at most 64 (32 warps per SM; 512 x 8 and
                                 1024 x 4, aggregate = 0);
                                 policy-capable kernels: 0 or 1 */
} ks_launch;

/*
 * Batched plans for uneven ensembles.  Each market belongs to the first
 * bucket (in plan order) with L <= L_max and A <= A_max.  A bucket's markets
 * run on groups of group_threads threads holding agents_per_thread agents
 * each; several groups share one CTA of cta_threads threads when they fit
 * (markets per CTA = min(cta_threads / group_threads, shared-memory fit)).
 * Work items (the markets one CTA runs together) are taken longest first
 * from a device ticket counter by the single persistent launch.
 */
typedef struct ks_bucket {
  int32_t L_max;
  int32_t A_max;
  int32_t group_threads;      /* a (group_threads, agents_per_thread) pair listed by ks_batch_variants */
  int32_t agents_per_thread;
} ks_bucket;

typedef struct ks_batch_info {
  int32_t batched;       /* 1 = the batched kernel runs ks_step_n                  */
  int32_t cta_threads;
  int32_t n_items;       /* work items (batched) or markets (plain)                */
  int32_t n_buckets;
  int32_t grid;          /* persistent CTAs launched                               */
  int32_t pad_;
  int64_t smem_bytes;    /* dynamic shared memory per CTA                          */
} ks_batch_info;

/* Bytes of device workspace needed for `cfg`. */
ks_status ks_workspace_size(const ks_config* cfg, size_t* bytes);

/* Validates cfg, lays out the ensemble in `workspace` (device, caller-owned,
 * 256-byte aligned, at least ks_workspace_size bytes, alive until
 * ks_destroy) and queues the init kernel on `stream` (step counter 0, every
 * market at price L/2 with empty books and zero accounts).  Returns a handle
 * in *out.  Chooses a default launch shape (see ks_set_launch). */
ks_status ks_create_ensemble(const ks_config* cfg, void* workspace, size_t ws_bytes, void* stream,
                             ks_ensemble** out);

/* Queues steps [s, s + n_steps) of every market on `stream`, where s is the
 * ensemble's step counter, then advances the counter on the device.  The
 * counter lives in device memory, so a CUDA graph captured around this call
 * continues the simulation on every replay.  Asynchronous; no allocation, no
 * host synchronisation (capturable). */
ks_status ks_step_n(ks_ensemble* e, uint32_t n_steps, void* stream);

/* Copies the requested fields into `dst` after the work queued on `stream`,
 * then synchronises `stream`. */
ks_status ks_read_state(ks_ensemble* e, const ks_state_view* dst, void* stream);

/* Overwrites the given fields from `src` (resume from a checkpoint made by
 * ks_read_state).  Queued on `stream`, then synchronised. */
ks_status ks_write_state(ks_ensemble* e, const ks_state_view* src, void* stream);

/* Waits for `stream` with a host-side deadline (0 = no deadline), then checks
 * the device error word: KS_ERR_TIMEOUT if the deadline passed (the GPU work
 * keeps running), KS_ERR_DEVICE_FAULT if a kernel reported an error. */
ks_status ks_sync(ks_ensemble* e, void* stream, uint32_t timeout_ms);

/* Device error word (0 = none) after synchronising `stream`. */
ks_status ks_error_word(ks_ensemble* e, void* stream, uint32_t* word);

/* Sets / gets the plain persistent kernel's launch shape (one market per CTA,
 * markets dealt round-robin).  ks_set_launch switches the ensemble to the
 * plain kernel.  When threads * agents_per_thread exceeds the ensemble's
 * largest A (and no warp aggregation is asked for), the launch runs the
 * shape's spreading variant where one is compiled: each market spreads its
 * agents over the CTA, ceil(A / threads) per thread; the results are the
 * same bit for bit.  Otherwise, for an ensemble that carries its book, a full
 * shape of the 128-register class (reg_cap 1; 128, 256 or 512 threads x 8 or
 * 16 agents) runs the kernel compiled for carried books, again with the same
 * results. */
ks_status ks_set_launch(ks_ensemble* e, const ks_launch* l);
ks_status ks_get_launch(const ks_ensemble* e, ks_launch* l);

/* Switches the ensemble to the batched kernel with the given plan; uploads the
 * work list on `stream` and synchronises it.  cta_threads: 512 or 1024.
 * Uneven ensembles start with a default plan: one bucket per power-of-two
 * (L, A) class and 512-thread CTAs.  Rule-agent buckets up to A = 512 take
 * 128 threads x 4 agents, up to 2048 A/8 threads x 8 (at least 128), up to
 * 8192 A/16 x 16, above that 512 x 32; policy buckets take the tightest
 * compiled fit near 8 agents per thread.  A market spreads its agents over
 * its group, ceil(A / group_threads) consecutive agents per thread; results
 * do not depend on the plan. */
ks_status ks_set_batch_plan(ks_ensemble* e, int32_t cta_threads, const ks_bucket* buckets, int32_t n_buckets,
                            void* stream);

/* The launch the next ks_step_n will make. */
ks_status ks_get_batch_info(const ks_ensemble* e, ks_batch_info* info);

/* (group_threads, agents_per_thread) pairs compiled into the batched kernel of
 * `cta_threads` threads: writes up to `capacity` pairs to `pairs` (may be
 * NULL) and their number to *count. */
ks_status ks_batch_variants(int32_t cta_threads, int32_t* pairs, int32_t capacity, int32_t* count);

/* Frees the host handle.  The workspace stays the caller's. */
ks_status ks_destroy(ks_ensemble* e);

/*
 * The paper's own agent model on a tick-aggregated book (Sec. III-C, "Agent
 * Decision and Order Aggregation"; Algorithm 1).  A second ensemble type: no
 * agent accounts and no cancellation.  Every step, every agent submits one
 * order; the step's orders clear (Eq. 1-2, ties as tie_rule, allocation in
 * price priority as above); their unfilled part is the resting book, whose
 * best bid bb and best ask ba give the next step's mid price (state
 * retrieval, Sec. III-C: mid = (bb + ba) / 2 when both exist, else the last
 * clearing tick).  The opening book is empty and the opening price L/2.
 * Agents (class from the channel-2 draw of step 0: MAKER if its percentile
 * floor(100 w / 2^32) < maker_pct, MOMENTUM if < maker_pct + mom_pct, else
 * NOISE):
 *  - NOISE: buys or sells with probability 1/2; with probability P_mkt a
 *    marketable order at tick L-1 (buy) or 0 (sell), else at round(mid + eta),
 *    eta uniform on [-noise_halfwidth, noise_halfwidth];
 *  - MOMENTUM: side = sign of the mid change since the previous step (the
 *    coin when zero; the first step's previous mid is L/2); marketable with
 *    probability P_mkt, else at round(mid + 1) (buy) / round(mid - 1) (sell);
 *  - MAKER: buys iff (a + s) mod 2 = 0, at round(mid - maker_half_spread),
 *    sells at round(mid + maker_half_spread); never marketable.
 * Quantity 1 + floor(qmax u).  round() is to the nearest integer with ties to
 * even; ticks are clamped to [0, L).
 * Draws (SplitMix64, Sec. III-G): u(gid, s, c) = mix64(seed +
 * 0x9E3779B97F4A7C15 * (gid * 2^35 + 8 s + c)), the output number
 * gid * 2^35 + 8 s + c of the generator with state `seed`, gid = (market_base
 * + m) * A + a.  Channel 0: high word = marketable draw (marketable iff below
 * p_mkt_q32), low word = side coin (sell iff >= 2^31); channel 1: high word =
 * price draw w (eta = -D + 2 D w / 2^32), low word = quantity draw (u =
 * w / 2^32); channel 2 at step 0: high word = class draw.
 * Sliding window (Sec. III-A; window = 1): the L ticks are a window onto an
 * unbounded grid, absolute tick = window_base + window tick, window_base 0 at
 * creation.  At the start of a step, once the mid is known, the window moves
 * if the mid is more than L/4 from its centre L/2 (integer part): by
 * k = 2 floor((2 mid - 2 (L/2)) / 4) ticks, an even number (so ties-to-even
 * rounding is the same in both coordinates), which puts the mid back within
 * one tick of the centre; the mid and the last price move with it.  Orders
 * beyond the window are clamped to its edges, marketable orders go to them.
 * The trace then records the absolute last price after each step (carried
 * on steps without trade); sum_price and the trace hash take absolute p*.
 */
typedef struct ks_paper_config {
  uint32_t n_markets;          /* M >= 1                                          */
  uint32_t market_base;        /* global index of market 0 (draws use it)         */
  int32_t L;                   /* ticks, 2..KS_MAX_TICKS                          */
  int32_t A;                   /* agents per market, 0..KS_MAX_AGENTS             */
  uint64_t seed;               /* SplitMix64 generator state                     */
  int32_t noise_halfwidth;     /* Delta_noise in ticks, 0..L                      */
  uint32_t p_mkt_q32;          /* P_mkt * 2^32                                    */
  int32_t qmax;                /* q_max, 1..KS_MAX_QTY                            */
  int32_t maker_half_spread;   /* Delta_maker_half_spread in ticks, 0..L          */
  uint32_t mom_pct;            /* alpha_mom in percent                            */
  uint32_t maker_pct;          /* alpha_maker in percent, mom_pct + maker_pct <= 100 */
  int32_t tie_rule;            /* ks_tie_rule                                     */
  uint32_t trace_markets;      /* markets 0..trace_markets-1 record (p*, V*) per step */
  uint32_t trace_steps;        /* trace capacity in steps                         */
  int32_t window;              /* 0: fixed grid; 1: sliding window (see above)    */
} ks_paper_config;

typedef struct ks_paper_ensemble ks_paper_ensemble;

/* State of a paper-agent ensemble (caller-owned buffers, host or device; NULL
 * fields are skipped). */
typedef struct ks_paper_state_view {
  int32_t* bid;          /* [M*L] resting buy quantity per tick: bid[m*L + p]  */
  int32_t* ask;          /* [M*L] resting sell quantity per tick               */
  int32_t* last_tick;    /* [M] last clearing tick                             */
  int32_t* mid2;         /* [M] twice the mid price of the latest step         */
  int32_t* trades;       /* [M] steps with V* > 0                              */
  int32_t* last_volume;  /* [M] V* of the latest step                          */
  int64_t* sum_price;    /* [M] sum of p* over trading steps                   */
  int64_t* sum_volume;   /* [M] sum of V* over steps                           */
  uint64_t* trace_hash;  /* [M] as ks_state_view::trace_hash (absolute p*)     */
  uint64_t* step;        /* [1] absolute step counter                          */
  int32_t* trace;        /* [trace_markets*trace_steps*2] (p*, V*) per market and step;
                            with a window, (absolute last price after the step, V*) */
  int64_t* window_base;  /* [M] absolute tick of window tick 0 (0 on a fixed grid) */
} ks_paper_state_view;

/* Workspace bytes, creation (init kernel queued on `stream`), steps [s, s+n)
 * in one persistent launch (asynchronous, capturable), state copies (then
 * `stream` is synchronised), launch shape, deadline wait and error word
 * check, handle release: as the functions above of the same name.  Launch
 * shape: `threads` per market (16: half a warp per market, eight markets
 * per 128-thread CTA, agents_per_thread 1, 2 or 4; 32: one warp per market,
 * four markets per 128-thread CTA, agents_per_thread 1, 2, 4, 8, 16 or 32;
 * 64: agents per thread 4 or 8; 128, 256: agents per thread 1..16; 512,
 * 1024: 16), threads *
 * agents_per_thread >= A; min_ctas 0 or 1 = the compiler's register choice,
 * else the register cap of min_ctas resident CTAs per SM (compiled: 16 x 2,
 * 16 x 4, 32 x 1, 32 x 2, 128 x 1 and 128 x 2 at 8; 32 x 8, 128 x 4 and
 * 128 x 8 at 6). */
ks_status ks_paper_workspace_size(const ks_paper_config* cfg, size_t* bytes);
ks_status ks_paper_create(const ks_paper_config* cfg, void* workspace, size_t ws_bytes, void* stream,
                          ks_paper_ensemble** out);
ks_status ks_paper_step_n(ks_paper_ensemble* e, uint32_t n_steps, void* stream);
/* The naive engine of the paper's work-depth comparison and ablation (Sec.
 * III-F, Sec. IV-I): steps [s, s+n) of the same ensemble as n launches of one
 * thread per market, the book kept in global memory (the resting rows are read
 * and the residual written back every step) and clearing by one serial sweep.
 * Same model and draws as ks_paper_step_n, so the two give bit-identical state
 * and may be mixed on one ensemble.  Asynchronous on `stream`; no shape limit
 * on A beyond the configuration's. */
ks_status ks_paper_step_n_naive(ks_paper_ensemble* e, uint32_t n_steps, void* stream);
ks_status ks_paper_read_state(ks_paper_ensemble* e, const ks_paper_state_view* dst, void* stream);
ks_status ks_paper_set_launch(ks_paper_ensemble* e, int32_t threads, int32_t agents_per_thread, int32_t min_ctas);
ks_status ks_paper_get_launch(const ks_paper_ensemble* e, int32_t* threads, int32_t* agents_per_thread,
                              int32_t* min_ctas);
ks_status ks_paper_sync(ks_paper_ensemble* e, void* stream, uint32_t timeout_ms);
ks_status ks_paper_destroy(ks_paper_ensemble* e);

const char* ks_status_string(ks_status s);
const char* ks_last_error(void);

/*
 * Agent policy (learned agents).  A 32 -> 64 -> 64 -> 37 ReLU network: logits
 * 0-2 are the side (buy, sell, pass), 3-35 the tick offset k = -16..+16 from
 * the last clearing tick counted toward the opposite side (a buy at last + k,
 * a sell at last - k), 36 the log-quantity.  Parameter blob (device memory,
 * 16-byte aligned, KS_MLP_PARAM_BYTES bytes):
 *   offset     0: W1 bf16 [64][32]  (row = output unit, column = input)
 *   offset  4096: W2 bf16 [64][64]
 *   offset 12288: W3 bf16 [37][64]
 *   offset 17024: b1 f32 [64], 17280: b2 f32 [64], 17536: b3 f32 [37]
 * Inputs (fp32): the last eight clearing-tick returns / 8 (newest first), the
 * agent's inventory / 256, the market's last executed volume / (8 A), resting
 * sell quantity at ticks last+1..last+4 and buy quantity at last-1..last-4,
 * each / (4 A), then 14 zeros.
 */
#define KS_MLP_PARAM_BYTES 17696

/*
 * Captures (learned-agent workflows; device buffers owned by the caller).
 *  - Rule-decision records, the behaviour-cloning data: every new order of a
 *    rule agent with index a < record_agents is appended as
 *    KS_RECORD_WORDS int32: the policy's 18 raw inputs (eight clearing-tick
 *    returns, newest first; inventory; last executed volume; resting sell
 *    quantity at last+1..+4; resting buy quantity at last-1..-4), side,
 *    offset index (the tick offset toward the opposite side, tick - last for
 *    a buy and last - tick for a sell, clamped to [-16, 16], plus 16), qty,
 *    agent class.  Records are appended in no particular order; *record_count
 *    counts every attempt, records beyond `record_capacity` are dropped.
 *  - Policy decisions of the traced markets: decisions[s * traced_agents + g]
 *    for absolute step s < trace_steps and global agent id g of a market
 *    m < trace_markets: an order word (qty, side, tick) of the order the
 *    policy placed, KS_DECISION_PASS if it passed, untouched if the agent made
 *    no policy decision at step s.
 */
#define KS_RECORD_WORDS 22
#define KS_DECISION_PASS 0x01000000u
typedef struct ks_capture {
  int32_t* records;
  uint64_t record_capacity;
  uint32_t record_agents;
  uint32_t pad_;
  unsigned long long* record_count;
  uint32_t* decisions;
  unsigned long long* policy_count;  /* device counter += policy decisions evaluated (NULL = off) */
  /* FP32 logits of every policy decision of the traced markets, [trace_steps]
   * [agents of the traced markets][37], indexed like `decisions` (absolute
   * step, ensemble agent index); entries without a decision are left as they
   * are (NULL = off; needs trace_markets and trace_steps). */
  float* logits;
} ks_capture;

/* Sets the ensemble's captures (NULL fields switch a capture off).  Capturing
 * runs the policy-capable kernels. */
ks_status ks_set_capture(ks_ensemble* e, const ks_capture* c);

/* Logits Z [n][37] (fp32) of feature rows X [n][32] (fp32), all device
 * pointers: layer 1 in FP32, layers 2-3 on the BF16 tcgen05 path the step
 * loop uses (BF16 weights, activations passed as high + low BF16 parts,
 * FP32 accumulation).  `err` (device uint32) receives error bits (a bounded
 * tensor-core wait that gave up). */
ks_status ks_mlp_forward(const void* params, const float* X, int64_t n, float* Z, uint32_t* err, void* stream);

/*
 * ks_step_n for callers that cannot allocate device memory for the batched
 * kernel's scratch.  The paper has no counterpart: this is a deployment
 * variant of the batched launch.
 *
 * ks_step_n keeps the batched kernel's scratch -- its work schedule (markets
 * grouped into work items, longest first) and the ticket counter the CTAs
 * take items from -- in the caller's workspace.  This entry point runs the
 * same kernel with that scratch in a static device array owned by the
 * library instead, of fixed size (KS_NOALLOC_MAX_MARKETS markets: about
 * 640 KB), which every GPU that loads the library holds until the process
 * exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
 *  - The ensemble must run the batched kernel (an uneven ensemble, or any
 *    ensemble after ks_set_batch_plan): else KS_ERR_INVALID_ARG.
 *  - More than KS_NOALLOC_MAX_MARKETS markets: KS_ERR_UNSUPPORTED.
 *  - The ensemble's device must be current: else KS_ERR_INVALID_ARG.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and keeps it for the life of the process; the
 *    entry point does not survive a cudaDeviceReset of that device.
 *  - Every call shares the array and overwrites it (it clears the ticket and
 *    copies the schedule from pageable host memory on `stream` before the
 *    launch), so calls that overlap on the GPU, on any streams, race.
 *  - A call on a stream that is being captured returns KS_ERR_UNSUPPORTED:
 *    the host copy of the schedule cannot be recorded safely.
 * Otherwise as ks_step_n: steps [s, s + n_steps), results identical.
 */
#define KS_NOALLOC_MAX_MARKETS 32768
ks_status ks_step_n_noalloc(ks_ensemble* e, uint32_t n_steps, void* stream);

/*
 * Behaviour-cloning training of the policy (hand-written kernels: the
 * contractions on the tensor cores as BF16 high + low parts with FP32
 * accumulation, the loss and Adam in FP32).
 * Parameter vector (FP32, device, KS_MLP_NPARAM floats):
 *   W1[64][32], b1[64], W2[64][64], b2[64], W3[37][64], b3[37].
 * Samples are rule-decision records (KS_RECORD_WORDS int32 each, see
 * ks_capture) of markets with A agents; the inputs are normalised as in the
 * step loop.  Per-sample loss: cross-entropy of the side (label record[18]),
 * cross-entropy of the offset index (record[19]) and the squared error of the
 * log-quantity (log record[20]).
 */
#define KS_MLP_NPARAM 8677

/* Device workspace (bytes) that ks_bc_grad needs for n samples on the
 * current device: one partial gradient per CTA. */
ks_status ks_bc_workspace_size(int64_t n, size_t* bytes);

/* grad += scale * d(sum of per-sample losses)/d params; *loss += scale * sum of
 * the losses (both device FP32; the caller zeroes them).  `workspace` is a
 * caller-owned device buffer of at least ks_bc_workspace_size(n) bytes
 * (KS_ERR_WORKSPACE_TOO_SMALL otherwise).  Deterministic: the same inputs on
 * the same device give the same gradient and loss bit for bit (fixed tile
 * assignment, fixed-order sums, no floating-point atomics). */
ks_status ks_bc_grad(const float* params, const int32_t* records, int64_t n, int32_t A, float* grad, float* loss,
                     float scale, void* workspace, size_t ws_bytes, void* stream);

/* One Adam update (Kingma and Ba, 2015) with bias correction for step >= 1;
 * m and v are the moment vectors; zeroes grad. */
ks_status ks_adam_step(float* params, float* grad, float* m, float* v, int32_t step, float lr, float beta1,
                       float beta2, float eps, void* stream);

/* Writes the policy blob the step loop reads (BF16 weights, FP32 biases). */
ks_status ks_mlp_export(const float* params, void* blob, void* stream);

/*
 * Continuous double auction (CDA).  The paper clears by a per-step call
 * auction and names the continuous double auction as a market the same
 * persistent, state-carrying pattern extends to (Discussion and
 * Limitations; Conclusion and Future Work).  This ensemble keeps the main
 * model's agents, draws, one working order per agent, per-order
 * cancellation and accounts, and replaces the batch clearing by continuous
 * matching.  Each step of a market:
 *  1. every working order is cancelled iff its step-s draw word w0 is below
 *     cancel_thresh_q32;
 *  2. every agent without a working order decides from the step-start
 *     state with the rule of the main model (zero intelligence, momentum,
 *     mean reversion);
 *  3. the new orders arrive one by one in ascending agent index; each
 *     trades at once against the opposite side in price-time priority (best
 *     price first, at one price the earliest arrival first), every fill at
 *     the resting order's tick, while its limit still crosses; the
 *     remainder rests behind the orders already at its tick;
 *  4. each fill moves the buyer's and the seller's inventory and cash at the
 *     fill's tick;
 *  5. the last clearing tick becomes the tick of the step's last fill
 *     (unchanged without fills); the trace records (that tick or -1, the
 *     step's volume), which the trace hash folds as in ks_state_view.
 * One warp runs one market at a time with the book in shared memory: a FIFO
 * of resting agents per (side, tick) and a bitmap of the nonempty ticks per
 * side.  Uniform markets; 2 <= L <= KS_MAX_TICKS, 0 <= A <= KS_CDA_MAX_AGENTS
 * (KS_ERR_UNSUPPORTED beyond, or when one market's book does not fit the
 * shared memory of a CTA).  The configuration's policy agents are not part
 * of this model.
 */
#define KS_CDA_MAX_AGENTS 8192
typedef struct ks_cda_config {
  uint32_t n_markets;          /* M                                                  */
  uint32_t market_base;        /* global index of market 0 (draws use it)           */
  int32_t L;                   /* ticks                                              */
  int32_t A;                   /* agents per market                                  */
  uint64_t seed;
  uint32_t cancel_thresh_q32;  /* per-order cancellation probability x 2^32          */
  uint32_t mix_pct[3];         /* zero intelligence / momentum / mean reversion, sum 100 */
  int32_t zi_offset, zi_qmax, mom_lookback, mom_offset_max, mr_offset_max, rb_qmax;
                               /* as ks_config (offsets 0..2047, quantities 1..255)  */
  uint32_t trace_markets;      /* leading markets that record a per-step trace       */
  uint32_t trace_steps;
} ks_cda_config;

typedef struct ks_cda_ensemble ks_cda_ensemble;

/* State of a CDA ensemble (caller-owned host buffers; NULL fields skipped). */
typedef struct ks_cda_state_view {
  uint32_t* order;       /* [N] order words as ks_state_view::order              */
  int32_t* inventory;    /* [N]                                                    */
  int64_t* cash;         /* [N]                                                    */
  int32_t* next;         /* [N] the agent resting next at the same side and tick
                            (time priority), -1 for the last one and for agents
                            without a resting order                             */
  int32_t* last_tick;    /* [M] last clearing tick                                 */
  int32_t* history;      /* [M*KS_HISTORY] newest first                           */
  int32_t* fundamental;  /* [M]                                                    */
  int32_t* fills;        /* [M] fills so far                                       */
  int32_t* last_volume;  /* [M] volume of the latest step                          */
  int64_t* traded_value; /* [M] sum over fills of tick * quantity                  */
  int64_t* sum_volume;   /* [M]                                                    */
  uint64_t* trace_hash;  /* [M]                                                    */
  uint64_t* step;        /* [1] absolute step counter                              */
  int32_t* trace;        /* [trace_markets*trace_steps*2] (last fill tick or -1, volume) */
} ks_cda_state_view;

/* Workspace bytes; creation in a caller-owned device workspace (initial state
 * as ks_create_ensemble: no resting orders, opening tick L/2; queued on
 * `stream`); steps [s, s+n) in one persistent launch (asynchronous); state
 * copies to host (then `stream` is synchronised); deadline wait and error
 * word check; handle release.  Errors as the functions of ks_config. */
ks_status ks_cda_workspace_size(const ks_cda_config* cfg, size_t* bytes);
ks_status ks_cda_create(const ks_cda_config* cfg, void* dev_workspace, size_t ws_bytes, void* cuda_stream,
                        ks_cda_ensemble** out);
ks_status ks_cda_step_n(ks_cda_ensemble* e, uint32_t n_steps, void* cuda_stream);
ks_status ks_cda_read_state(ks_cda_ensemble* e, const ks_cda_state_view* dst, void* cuda_stream);
ks_status ks_cda_sync(ks_cda_ensemble* e, void* cuda_stream, uint32_t timeout_ms);
ks_status ks_cda_destroy(ks_cda_ensemble* e);

/* Library version, e.g. 0x000100 for 0.1.0. */
uint32_t ks_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KINETICSIM_H */
