// ks_capi.cu -- the C ABI of kineticsim.h: validation, workspace layout,
// ensemble initialisation, persistent-kernel launches and state I/O.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <thread>
#include <vector>

#include "kineticsim.h"
#include "kineticsim_probe.h"
#include "ks_device.cuh"
#include "ks_internal.h"
#include "ks_batched.cuh"
#include "ks_plain.cuh"

namespace ks {
extern const PlainVariant kPlainNT128[];
extern const PlainVariant kPlainNT256[];
extern const PlainVariant kPlainNT512[];
extern const PlainVariant kPlainNT1024[];
extern const int kPlainNT128Count, kPlainNT256Count, kPlainNT512Count, kPlainNT1024Count;
extern const PlainVariant kPlainSpreadA[];
extern const PlainVariant kPlainSpreadB[];
extern const PlainVariant kPlainCarried[];
extern const int kPlainCarriedCount;
extern const int kPlainSpreadACount, kPlainSpreadBCount;
extern const int kBatchVariants512[][2];
extern const int kBatchVariants1024[][2];
extern const int kBatchVariants512Count, kBatchVariants1024Count;
cudaError_t launch_batched_512(const DevParams& p, uint32_t n_steps, const BatchArgs& b, int grid, size_t smem,
                               cudaStream_t st);
cudaError_t launch_batched_1024(const DevParams& p, uint32_t n_steps, const BatchArgs& b, int grid, size_t smem,
                                cudaStream_t st);
const void* batched_kernel_512();
const void* batched_kernel_1024();
extern const PlainVariant kPlainMlp[];
extern const int kPlainMlpCount;
extern const int kBatchMlpVariants512[][2];
extern const int kBatchMlpVariants512Count;
cudaError_t launch_batched_mlp_512(const DevParams& p, uint32_t n_steps, const BatchArgs& b, int grid, size_t smem,
                                   cudaStream_t st);
const void* batched_mlp_kernel_512();

const PlainVariant* find_plain(int threads, int ak, int aggregate, int occupancy, bool mlp) {
  if (mlp) {
    for (int j = 0; j < kPlainMlpCount; ++j)
      if (kPlainMlp[j].threads == threads && kPlainMlp[j].ak == ak && kPlainMlp[j].occupancy == occupancy)
        return &kPlainMlp[j];
    return nullptr;
  }
  const PlainVariant* tabs[4] = {kPlainNT128, kPlainNT256, kPlainNT512, kPlainNT1024};
  const int counts[4] = {kPlainNT128Count, kPlainNT256Count, kPlainNT512Count, kPlainNT1024Count};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < counts[i]; ++j) {
      const PlainVariant& v = tabs[i][j];
      if (v.threads == threads && v.ak == ak && v.aggregate == (aggregate ? 1 : 0) && v.occupancy == occupancy)
        return &v;
    }
  return nullptr;
}

const PlainVariant* find_plain_spread(int threads, int ak, int occupancy) {
  const PlainVariant* tabs[2] = {kPlainSpreadA, kPlainSpreadB};
  const int counts[2] = {kPlainSpreadACount, kPlainSpreadBCount};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < counts[i]; ++j) {
      const PlainVariant& v = tabs[i][j];
      if (v.threads == threads && v.ak == ak && v.occupancy == occupancy) return &v;
    }
  return nullptr;
}

const PlainVariant* find_plain_carried(int threads, int ak, int occupancy) {
  for (int j = 0; j < kPlainCarriedCount; ++j) {
    const PlainVariant& v = kPlainCarried[j];
    if (v.threads == threads && v.ak == ak && v.occupancy == occupancy) return &v;
  }
  return nullptr;
}

static const int (*batch_table(int nt, int* count, bool mlp = false))[2] {
  if (mlp) {
    if (nt == 512) {
      *count = kBatchMlpVariants512Count;
      return kBatchMlpVariants512;
    }
    *count = 0;  // the policy batched kernel is compiled for 512-thread CTAs only
    return nullptr;
  }
  if (nt == 512) {
    *count = kBatchVariants512Count;
    return kBatchVariants512;
  }
  if (nt == 1024) {
    *count = kBatchVariants1024Count;
    return kBatchVariants1024;
  }
  *count = 0;
  return nullptr;
}

// ---------------------------------------------------------------------------
// Initial state (the paper's Phase 1: empty book, opening price L/2).
// ---------------------------------------------------------------------------
__global__ void init_kernel(DevParams P) {
  for (uint32_t m = blockIdx.x; m < P.M; m += gridDim.x) {
    const int L = P.Ls ? P.Ls[m] : P.L_all;
    const int A = P.As ? P.As[m] : P.A_all;
    const int64_t off = P.agent_off ? P.agent_off[m] : (int64_t)m * P.A_all;
    for (int a = threadIdx.x; a < A; a += blockDim.x) {
      const uint4 w = philox(0u, (uint32_t)a, P.market_base + m, 1u, P.key0, P.key1);
      const uint32_t pct = __umulhi(w.x, 100u);
      const uint32_t cls = pct < P.mix0 ? KS_CLASS_ZI : (pct < P.mix01 ? KS_CLASS_MOM : KS_CLASS_MR);
      const bool mlp = __umulhi(w.y, 100u) < P.mlp_pct;
      P.slot[off + a] = (cls << W_CLASS_SHIFT) | (mlp ? W_MLP : 0u);
      P.inv[off + a] = 0;
      P.cash[off + a] = 0;
    }
    if (threadIdx.x == 0) {
      int32_t* mi = P.mi32 + (size_t)m * MI32_STRIDE;
      mi[MI_LAST] = L / 2;
      for (int j = 0; j < KS_HISTORY; ++j) mi[MI_HIST + j] = L / 2;
      const uint4 w = philox(0u, 0u, P.market_base + m, 2u, P.key0, P.key1);
      mi[MI_FUND] = L / 4 + (int)__umulhi(w.x, (uint32_t)(L / 2 + 1));
      mi[MI_TRADES] = 0;
      mi[MI_LASTV] = 0;
      mi[13] = mi[14] = mi[15] = 0;
      int64_t* m64 = P.mi64 + (size_t)m * MI64_STRIDE;
      m64[0] = m64[1] = m64[2] = m64[3] = 0;
    }
  }
}

// Advances the device step counter after a launch and re-arms the batched
// kernel's work ticket for the next launch.
__global__ void step_bump_kernel(uint64_t* step, uint32_t* ticket, uint32_t n) {
  *step += n;
  *ticket = 0u;
}

}  // namespace ks

using namespace ks;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local char g_last_error[512] = "";

namespace ks {
// Error text for ks_last_error from the other translation units of the library.
void internal_set_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
}  // namespace ks

static ks_status cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return KS_ERR_CUDA;
}
#define KS_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

static ks_status arg_fail(ks_status s, const char* msg) {
  snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
  return s;
}

// ---------------------------------------------------------------------------
// Handle and workspace layout
// ---------------------------------------------------------------------------
struct ks_ensemble {
  ks_config cfg;
  uint32_t M;
  int64_t N;
  int Lmax, Amax;
  bool uniform;
  std::vector<int32_t> L, A;
  std::vector<int64_t> off;
  unsigned char* ws;
  size_t ws_bytes;
  DevParams dp;
  int mode;  // 0 plain kernel, 1 batched kernel
  ks_launch launch;
  const PlainVariant* var;
  int grid;
  size_t smem;
  // batched mode
  int b_threads;
  std::vector<ks_bucket> b_plan;
  std::vector<uint32_t> b_order;
  std::vector<uint4> b_items;
  BatchArgs b_args;
  int b_grid;
  size_t b_smem;
  int device;
  int num_sms;
  size_t max_smem;
  bool mlp;  // the policy-capable kernels run (policy agents or captures)
};

struct Layout {
  size_t slot, inv, cash, mi32, mi64, aoff, Ls, As, order, items, trace, ctrl, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static Layout make_layout(uint32_t M, int64_t N, bool uniform, uint32_t tm, uint32_t ts) {
  Layout l;
  size_t o = 0;
  l.slot = o; o = align256(o + (size_t)N * 4);
  l.inv = o; o = align256(o + (size_t)N * 4);
  l.cash = o; o = align256(o + (size_t)N * 8);
  l.mi32 = o; o = align256(o + (size_t)M * MI32_STRIDE * 4);
  l.mi64 = o; o = align256(o + (size_t)M * MI64_STRIDE * 8);
  l.aoff = o; o = align256(o + (uniform ? 0 : (size_t)(M + 1) * 8));
  l.Ls = o; o = align256(o + (uniform ? 0 : (size_t)M * 4));
  l.As = o; o = align256(o + (uniform ? 0 : (size_t)M * 4));
  l.order = o; o = align256(o + (size_t)M * 4);
  l.items = o; o = align256(o + (size_t)M * 16);
  l.trace = o; o = align256(o + (size_t)tm * ts * 2 * 4);
  l.ctrl = o; o = align256(o + 64);  // err (u32) at +0, step (u64) at +8, ticket (u32) at +16
  l.total = o;
  return l;
}

struct Sizes {
  std::vector<int32_t> L, A;
  std::vector<int64_t> off;
  int Lmax = 0, Amax = 0;
  bool uniform = true;
  int64_t N = 0;
};

static ks_status validate(const ks_config* c, Sizes* sz) {
  if (!c) return arg_fail(KS_ERR_INVALID_ARG, "config is NULL");
  if (c->n_markets == 0) return arg_fail(KS_ERR_INVALID_ARG, "n_markets must be >= 1");
  if (c->n_markets > (1u << 26)) return arg_fail(KS_ERR_UNSUPPORTED, "n_markets above 2^26");
  if ((uint64_t)c->market_base + c->n_markets > 0xFFFFFFFFull)
    return arg_fail(KS_ERR_INVALID_ARG, "market_base + n_markets above 2^32");
  if (c->mix_pct[0] + c->mix_pct[1] + c->mix_pct[2] != 100u)
    return arg_fail(KS_ERR_INVALID_ARG, "mix_pct must sum to 100");
  if (c->zi_offset < 0 || c->zi_offset > KS_MAX_TICKS) return arg_fail(KS_ERR_INVALID_ARG, "zi_offset out of range");
  if (c->mom_offset_max < 0 || c->mom_offset_max > KS_MAX_TICKS || c->mr_offset_max < 0 ||
      c->mr_offset_max > KS_MAX_TICKS)
    return arg_fail(KS_ERR_INVALID_ARG, "offset max out of range");
  if (c->zi_qmax < 1 || c->rb_qmax < 1) return arg_fail(KS_ERR_INVALID_ARG, "qmax must be >= 1");
  if (c->zi_qmax > KS_MAX_QTY || c->rb_qmax > KS_MAX_QTY) return arg_fail(KS_ERR_UNSUPPORTED, "qmax above 255");
  if (c->mom_lookback < 1 || c->mom_lookback > KS_HISTORY - 1)
    return arg_fail(KS_ERR_INVALID_ARG, "mom_lookback must be in [1, 8]");
  if (c->tie_rule != KS_TIE_LOWEST_TICK && c->tie_rule != KS_TIE_MIN_IMBALANCE)
    return arg_fail(KS_ERR_INVALID_ARG, "unknown tie_rule");
  if (c->mlp_pct > 100u) return arg_fail(KS_ERR_INVALID_ARG, "mlp_pct above 100");
  if (c->mlp_pct > 0u && !c->mlp_params) return arg_fail(KS_ERR_INVALID_ARG, "mlp_pct > 0 needs mlp_params");
  if (c->mlp_params && ((uintptr_t)c->mlp_params & 15u) != 0)
    return arg_fail(KS_ERR_INVALID_ARG, "mlp_params not 16-byte aligned");
  if (c->trace_markets > c->n_markets) return arg_fail(KS_ERR_INVALID_ARG, "trace_markets above n_markets");
  if ((c->trace_markets == 0) != (c->trace_steps == 0) && c->trace_markets != 0)
    return arg_fail(KS_ERR_INVALID_ARG, "trace_steps must be > 0 when tracing");
  const uint32_t M = c->n_markets;
  sz->L.resize(M);
  sz->A.resize(M);
  sz->off.resize(M + 1);
  int64_t n = 0;
  for (uint32_t m = 0; m < M; ++m) {
    const int32_t L = c->L ? c->L[m] : c->L_all;
    const int32_t A = c->A ? c->A[m] : c->A_all;
    if (L < 2 || A < 0) return arg_fail(KS_ERR_INVALID_ARG, "L must be >= 2 and A >= 0");
    if (L > KS_MAX_TICKS || A > KS_MAX_AGENTS) return arg_fail(KS_ERR_UNSUPPORTED, "L or A above the envelope");
    sz->L[m] = L;
    sz->A[m] = A;
    sz->off[m] = n;
    n += A;
    sz->Lmax = std::max(sz->Lmax, (int)L);
    sz->Amax = std::max(sz->Amax, (int)A);
  }
  sz->off[M] = n;
  sz->N = n;
  sz->uniform = true;
  for (uint32_t m = 1; m < M; ++m)
    if (sz->L[m] != sz->L[0] || sz->A[m] != sz->A[0]) sz->uniform = false;
  return KS_OK;
}

static int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Default launch shape: with few markets, spread each market over many
// threads; otherwise 16 agents per thread under the 128-register cap, two
// 256-thread CTAs per SM (the fastest shape measured on GB300 for
// 4096-agent markets).
static ks_launch default_launch(int Amax, uint32_t M, int num_sms, bool mlp = false) {
  ks_launch l;
  memset(&l, 0, sizeof(l));
  if (mlp) {
    // the smallest compiled policy shape that holds the largest market;
    // among equal ones the 128-register cap (two CTAs per SM), then more
    // threads (measured on 2048-agent markets: 256 x 8 capped 3.4e10
    // events/s, uncapped 2.3e10, 128 x 16 capped 2.8e10)
    int best = -1;
    for (int j = 0; j < kPlainMlpCount; ++j) {
      const PlainVariant& v = kPlainMlp[j];
      if ((int64_t)v.threads * v.ak < Amax) continue;
      if (best < 0) {
        best = j;
        continue;
      }
      const PlainVariant& b = kPlainMlp[best];
      const int64_t cap = (int64_t)v.threads * v.ak, bcap = (int64_t)b.threads * b.ak;
      if (cap != bcap ? cap < bcap
                      : (v.occupancy != b.occupancy ? v.occupancy > b.occupancy : v.threads > b.threads))
        best = j;
    }
    if (best < 0) best = kPlainMlpCount - 1;
    l.threads = kPlainMlp[best].threads;
    l.agents_per_thread = kPlainMlp[best].ak;
    l.reg_cap = kPlainMlp[best].occupancy;
    return l;
  }
  const bool few = (int)M < 2 * num_sms;
  int nt = few ? next_pow2(std::max(Amax, 1)) : next_pow2((std::max(Amax, 1) + 15) / 16);
  nt = std::min(1024, std::max(128, nt));
  int ak = next_pow2(std::max(1, (Amax + nt - 1) / nt));
  while (ak > 16 && nt < 1024) {
    nt *= 2;
    ak = next_pow2(std::max(1, (Amax + nt - 1) / nt));
  }
  l.threads = nt;
  l.agents_per_thread = ak;
  l.ctas_per_sm = 0;
  l.aggregate = 0;
  l.reg_cap = few ? 0 : 1;
  return l;
}

// Resident CTAs per SM of a persistent kernel.  The runtime's occupancy
// calculator answers one CTA per SM for every kernel that contains tcgen05
// instructions (CUDA 13.0 on GB300), although the hardware runs several such
// CTAs on one SM at the same time (measured: up to five 256-thread CTAs,
// each holding 32 TMEM columns).  For those kernels (tmem_cols > 0) the count
// is taken here from the same limits -- threads, registers (256-register
// allocation granules per warp), shared memory with the per-CTA reservation,
// CTA slots -- and from the 512 TMEM columns of an SM.  An overestimate is
// harmless: CTAs beyond the resident ones start when others finish.
static cudaError_t resident_ctas(const void* k, int threads, size_t smem, int tmem_cols, int* occ) {
  if (tmem_cols <= 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, threads, smem);
  cudaFuncAttributes a;
  cudaError_t rc = cudaFuncGetAttributes(&a, k);
  if (rc != cudaSuccess) return rc;
  int dev = 0, max_thr = 0, max_regs = 0, max_smem = 0, reserved = 0, max_blocks = 0;
  if ((rc = cudaGetDevice(&dev)) != cudaSuccess) return rc;
  cudaDeviceGetAttribute(&max_thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&max_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if ((rc = cudaDeviceGetAttribute(&max_blocks, cudaDevAttrMaxBlocksPerMultiprocessor, dev)) != cudaSuccess) return rc;
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((std::max(a.numRegs, 1) * 32 + 255) / 256) * 256;
  int n = max_thr / (warps * 32);
  n = std::min(n, max_regs / (regs_warp * warps));
  n = std::min(n, (int)((size_t)max_smem / (smem + a.sharedSizeBytes + (size_t)reserved)));
  n = std::min(n, max_blocks);
  n = std::min(n, 512 / tmem_cols);
  *occ = std::max(n, 0);
  return cudaSuccess;
}

static ks_status apply_launch(ks_ensemble* e, const ks_launch* l) {
  const PlainVariant* v = find_plain(l->threads, l->agents_per_thread, l->aggregate, l->reg_cap, e->mlp);
  if (!v)
    return arg_fail(KS_ERR_INVALID_ARG, e->mlp ? "no policy-capable kernel for this (threads, agents_per_thread, reg_cap)"
                                               : "no kernel for this (threads, agents_per_thread, aggregate, reg_cap)");
  if ((int64_t)l->threads * l->agents_per_thread < e->Amax)
    return arg_fail(KS_ERR_INVALID_ARG, "threads * agents_per_thread below the largest A");
  // a shape with room to spare: the variant that spreads each market's agents
  // over the CTA, where one is compiled (same state bit for bit, fewer passes)
  if (!e->mlp && !l->aggregate && (int64_t)l->threads * l->agents_per_thread > e->Amax) {
    const PlainVariant* sv = find_plain_spread(l->threads, l->agents_per_thread, l->reg_cap);
    if (sv) v = sv;
  }
  // a full shape over carried books: the variant compiled for that book mode,
  // where one is compiled (1.1% on the 8192-market workload, same state)
  if (!e->mlp && !l->aggregate && !v->spread && e->dp.carry) {
    const PlainVariant* cv = find_plain_carried(l->threads, l->agents_per_thread, l->reg_cap);
    if (cv) v = cv;
  }
  if (l->ctas_per_sm < 0 || l->ctas_per_sm > 32) return arg_fail(KS_ERR_INVALID_ARG, "ctas_per_sm out of range");
  size_t smem = plain_launch_smem(l->threads, l->agents_per_thread, l->reg_cap, e->Lmax, e->mlp);
  if (smem > e->max_smem) return arg_fail(KS_ERR_UNSUPPORTED, "launch shape needs more shared memory than a CTA has");
  const void* k = v->kernel;
  KS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  int tile_wgs = 1;
  int tmem_cols = 0;
  if (e->mlp) {
    // as many warpgroups evaluate policy tiles (MLP_TMEM_COLS TMEM columns
    // each, a power of two in all) as the SM's 512 columns allow without
    // lowering the resident CTAs that the other limits give
    int occ0 = 0;
    KS_CUDA(resident_ctas(k, l->threads, smem, 32, &occ0));
    tile_wgs = std::min(l->threads / 128, (int)MLP_MAX_TILE_WGS);
    while (tile_wgs > 1 && occ0 * tile_wgs * (int)MLP_TMEM_COLS > 512) tile_wgs /= 2;
    tmem_cols = tile_wgs * (int)MLP_TMEM_COLS;
  }
  KS_CUDA(resident_ctas(k, l->threads, smem, tmem_cols, &occ));
  if (occ < 1) return arg_fail(KS_ERR_UNSUPPORTED, "launch shape does not fit on an SM");
  // resident CTAs must not ask for more TMEM than an SM has (512 columns)
  if (e->mlp && occ * tmem_cols > 512) return arg_fail(KS_ERR_UNSUPPORTED, "policy launch oversubscribes TMEM");
  const int per_sm = l->ctas_per_sm > 0 ? std::min(occ, l->ctas_per_sm) : occ;
  e->grid = (int)std::min<int64_t>((int64_t)e->M, (int64_t)per_sm * e->num_sms);
  e->smem = smem;
  e->dp.mlp_tile_wgs = tile_wgs;
  e->var = v;
  e->launch = *l;
  e->mode = 0;
  return KS_OK;
}

// ---------------------------------------------------------------------------
// Batched plans: buckets -> work items (markets per CTA, longest first)
// ---------------------------------------------------------------------------
static int batch_variant_id(int nt, int gt, int ak, bool mlp) {
  int n = 0;
  const int(*tab)[2] = batch_table(nt, &n, mlp);
  for (int i = 0; i < n; ++i)
    if (tab[i][0] == gt && tab[i][1] == ak) return i;
  return -1;
}

// Groups of one bucket that fit one CTA: thread count, barrier ids, shared
// memory (the policy kernels keep their activations in TMEM).
static int groups_per_cta(int nt, int gt, int ak, int Lcap, size_t max_smem, size_t* gsz, bool mlp) {
  size_t o[8];
  *gsz = group_smem_layout(thread_reg_budget(nt, 1), gt, ak, Lcap, mlp, o);
  if (mlp) max_smem = max_smem > mlp_cta_bytes() ? max_smem - mlp_cta_bytes() : 0;
  int g = nt / gt;
  if (gt != 32 && gt != nt) g = std::min(g, 15);
  g = std::min<int64_t>(g, (int64_t)(max_smem / *gsz));
  return g;
}

// Default bucket shape.  Rule-agent buckets spread a market over its group
// (ceil(A / threads) agents per thread), so spare capacity costs little: 8
// agents per thread up to A = 2048, 16 up to 8192, then 32, with at least 32
// threads (one warp, __syncwarp barriers).  With the clearing confined to the
// ticks that can hold orders, small groups no longer pay for wide grids:
// measured on the 20000-market ensemble this rule gives 1.37e11 agent-events/s
// against 1.32e11 for the earlier one (4 agents per thread up to A = 512, at
// least 128 threads).  Policy buckets take the same table with groups of at
// least one warpgroup (fewer agents per thread below 1024 agents): measured on
// the 32768-market 25%-policy ensemble (10000 steps), 4.00e10 against 3.87e10
// for the tightest fit at 8 agents per thread (512 x 8 for 4096 agents, where
// 256 x 16 runs two markets per CTA).  Shapes a CTA size does not compile take the
// tightest fit at about 8 agents per thread.
static bool default_shape(int nt, int Ac, int* gt, int* ak, bool mlp) {
  int n = 0;
  const int(*tab)[2] = batch_table(nt, &n, mlp);
  {
    // 8 agents per thread up to 2048 agents, 16 up to 8192, then 32; a group
    // is at least a warp (a warpgroup for the policy kernel, whose narrowest
    // groups then take fewer agents per thread)
    const int k0 = Ac <= 2048 ? 8 : (Ac <= 8192 ? 16 : 32);
    const int gmin = mlp ? 128 : 32;
    const int g = std::max(gmin, Ac / k0);
    const int k = mlp ? std::max(4, Ac / g) : k0;
    for (int i = 0; i < n; ++i)
      if (tab[i][0] == g && tab[i][1] == k && g <= nt) {
        *gt = g;
        *ak = k;
        return true;
      }
  }
  int best = -1;
  long best_score = 0;
  for (int i = 0; i < n; ++i) {
    const int g = tab[i][0], k = tab[i][1];
    if ((long)g * k < Ac) continue;
    const long waste = (long)g * k - Ac;
    const long score = waste * 16 + std::abs(k - 8);
    if (best < 0 || score < best_score) {
      best = i;
      best_score = score;
    }
  }
  if (best < 0) return false;
  *gt = tab[best][0];
  *ak = tab[best][1];
  return true;
}

// CTA size of the default batched plan (the policy-capable batched kernel exists for 512 only).
constexpr int kDefaultBatchThreads = 512;

static std::vector<ks_bucket> default_plan(const std::vector<int32_t>& L, const std::vector<int32_t>& A, int nt,
                                           bool mlp) {
  std::vector<std::pair<int, int>> keys;
  for (size_t m = 0; m < L.size(); ++m) {
    const int Lc = std::max(32, next_pow2(L[m]));
    const int Ac = std::max(32, next_pow2(std::max(A[m], 1)));
    keys.emplace_back(Lc, Ac);
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  std::vector<ks_bucket> plan;
  for (auto& k : keys) {
    ks_bucket b;
    b.L_max = k.first;
    b.A_max = k.second;
    if (!default_shape(nt, k.second, &b.group_threads, &b.agents_per_thread, mlp)) continue;
    plan.push_back(b);
  }
  return plan;
}

static ks_status build_batch(ks_ensemble* e, int nt, const ks_bucket* buckets, int nb, cudaStream_t st) {
  if (nt != 512 && nt != 1024) return arg_fail(KS_ERR_INVALID_ARG, "batched CTA size must be 512 or 1024");
  if (nb <= 0 || !buckets) return arg_fail(KS_ERR_INVALID_ARG, "empty batch plan");
  const bool mlp = e->mlp;
  if (mlp && nt != 512) return arg_fail(KS_ERR_INVALID_ARG, "the policy batched kernel uses 512-thread CTAs");
  const void* kern = mlp ? batched_mlp_kernel_512() : (nt == 512 ? batched_kernel_512() : batched_kernel_1024());
  const size_t max_dyn = e->max_smem - 1024;  // room for the kernel's static shared memory
  std::vector<int> var(nb);
  std::vector<int> G(nb);
  std::vector<size_t> gsz(nb);
  for (int b = 0; b < nb; ++b) {
    const ks_bucket& k = buckets[b];
    var[b] = batch_variant_id(nt, k.group_threads, k.agents_per_thread, mlp);
    if (var[b] < 0)
      return arg_fail(KS_ERR_INVALID_ARG, mlp ? "bucket shape not compiled into the policy batched kernel"
                                              : "bucket shape not compiled into the batched kernel");
    if ((int64_t)k.group_threads * k.agents_per_thread < k.A_max)
      return arg_fail(KS_ERR_INVALID_ARG, "bucket group_threads * agents_per_thread below its A_max");
    if (k.L_max < 2 || k.L_max > KS_MAX_TICKS) return arg_fail(KS_ERR_INVALID_ARG, "bucket L_max out of range");
    G[b] = groups_per_cta(nt, k.group_threads, k.agents_per_thread, k.L_max, max_dyn, &gsz[b], mlp);
    if (G[b] < 1) return arg_fail(KS_ERR_UNSUPPORTED, "bucket does not fit the shared memory of one CTA");
  }
  std::vector<std::vector<uint32_t>> members(nb);
  for (uint32_t m = 0; m < e->M; ++m) {
    int b = 0;
    while (b < nb && !(e->L[m] <= buckets[b].L_max && e->A[m] <= buckets[b].A_max)) ++b;
    if (b == nb) return arg_fail(KS_ERR_INVALID_ARG, "a market matches no bucket of the plan");
    members[b].push_back(m);
  }
  // policy kernel: every warpgroup of a group evaluates policy tiles (each
  // owns MLP_TMEM_COLS columns of the CTA's tensor memory)
  std::vector<int> tile_wgs(nb, 1);
  if (mlp)
    for (int b = 0; b < nb; ++b) tile_wgs[b] = std::max(1, buckets[b].group_threads / 128);
  struct Item {
    double cost;
    int bucket;
    std::vector<uint32_t> mk;
  };
  std::vector<Item> items;
  size_t smem = 16;
  for (int b = 0; b < nb; ++b) {
    auto& mb = members[b];
    if (mb.empty()) continue;
    std::sort(mb.begin(), mb.end(), [&](uint32_t x, uint32_t y) {
      return e->A[x] != e->A[y] ? e->A[x] > e->A[y] : x < y;
    });
    smem = std::max(smem, (size_t)std::min<size_t>(G[b], mb.size()) * gsz[b]);
    for (size_t i = 0; i < mb.size(); i += G[b]) {
      Item it;
      it.bucket = b;
      it.mk.assign(mb.begin() + i, mb.begin() + std::min(mb.size(), i + G[b]));
      // cost of an item ~ its largest market: agent work plus the per-step tick work
      it.cost = (double)e->A[it.mk[0]] + 0.25 * (double)buckets[b].L_max;
      items.push_back(std::move(it));
    }
  }
  std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.cost > y.cost; });
  if (mlp) smem += mlp_cta_bytes();
  std::vector<uint32_t> order;
  std::vector<uint4> ditems;
  for (auto& it : items) {
    uint4 d;
    d.x = (uint32_t)order.size();
    d.y = (uint32_t)it.mk.size();
    // variant id; the policy kernel also reads its tile warpgroups from bits 16+
    d.z = (uint32_t)var[it.bucket] | (mlp ? (uint32_t)tile_wgs[it.bucket] << 16 : 0u);
    d.w = (uint32_t)buckets[it.bucket].L_max;
    order.insert(order.end(), it.mk.begin(), it.mk.end());
    ditems.push_back(d);
  }
  KS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  KS_CUDA(resident_ctas(kern, nt, smem, mlp ? (nt / 128) * (int)MLP_TMEM_COLS : 0, &occ));
  if (occ < 1) return arg_fail(KS_ERR_UNSUPPORTED, "batched plan does not fit on an SM");
  if (mlp && occ * (nt / 128) * (int)MLP_TMEM_COLS > 512)
    return arg_fail(KS_ERR_UNSUPPORTED, "policy batched launch oversubscribes TMEM");
  const Layout lay = make_layout(e->M, e->N, e->uniform, e->cfg.trace_markets, e->cfg.trace_steps);
  KS_CUDA(cudaMemcpyAsync(e->ws + lay.order, order.data(), order.size() * 4, cudaMemcpyHostToDevice, st));
  KS_CUDA(cudaMemcpyAsync(e->ws + lay.items, ditems.data(), ditems.size() * 16, cudaMemcpyHostToDevice, st));
  KS_CUDA(cudaStreamSynchronize(st));  // the host vectors feeding the copies may be reused
  e->b_threads = nt;
  e->b_plan.assign(buckets, buckets + nb);
  e->b_order = std::move(order);
  e->b_items = std::move(ditems);
  e->b_args.order = (const uint32_t*)(e->ws + lay.order);
  e->b_args.items = (const uint4*)(e->ws + lay.items);
  e->b_args.n_items = (uint32_t)e->b_items.size();
  e->b_args.ticket = (uint32_t*)(e->ws + lay.ctrl + 16);
  e->b_smem = smem;
  e->b_grid = (int)std::min<int64_t>((int64_t)occ * e->num_sms, std::max<int64_t>(1, (int64_t)e->b_items.size()));
  e->mode = 1;
  return KS_OK;
}

static cudaError_t launch_main(ks_ensemble* e, uint32_t n_steps, cudaStream_t st) {
  if (e->mode == 1) {
    if (e->mlp) return launch_batched_mlp_512(e->dp, n_steps, e->b_args, e->b_grid, e->b_smem, st);
    return e->b_threads == 512 ? launch_batched_512(e->dp, n_steps, e->b_args, e->b_grid, e->b_smem, st)
                               : launch_batched_1024(e->dp, n_steps, e->b_args, e->b_grid, e->b_smem, st);
  }
  return e->var->launch(e->dp, n_steps, e->grid, e->smem, st);
}

// ---------------------------------------------------------------------------
// Public API
// ---------------------------------------------------------------------------
extern "C" {

uint32_t ks_version(void) { return 0x000100u; }

const char* ks_last_error(void) { return g_last_error; }

const char* ks_status_string(ks_status s) {
  switch (s) {
    case KS_OK: return "ok";
    case KS_ERR_INVALID_ARG: return "invalid argument";
    case KS_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case KS_ERR_CUDA: return "CUDA error";
    case KS_ERR_UNSUPPORTED: return "unsupported configuration";
    case KS_ERR_DEVICE_FAULT: return "device error word set";
    case KS_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

ks_status ks_workspace_size(const ks_config* cfg, size_t* bytes) {
  if (!bytes) return arg_fail(KS_ERR_INVALID_ARG, "bytes is NULL");
  Sizes sz;
  ks_status s = validate(cfg, &sz);
  if (s != KS_OK) return s;
  *bytes = make_layout(cfg->n_markets, sz.N, sz.uniform, cfg->trace_markets, cfg->trace_steps).total;
  return KS_OK;
}

ks_status ks_create_ensemble(const ks_config* cfg, void* workspace, size_t ws_bytes, void* stream,
                             ks_ensemble** out) {
  if (!out) return arg_fail(KS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  Sizes sz;
  ks_status s = validate(cfg, &sz);
  if (s != KS_OK) return s;
  if (!workspace) return arg_fail(KS_ERR_INVALID_ARG, "workspace is NULL");
  if (((uintptr_t)workspace & 255u) != 0) return arg_fail(KS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  const Layout lay = make_layout(cfg->n_markets, sz.N, sz.uniform, cfg->trace_markets, cfg->trace_steps);
  if (ws_bytes < lay.total) return arg_fail(KS_ERR_WORKSPACE_TOO_SMALL, "workspace smaller than ks_workspace_size");
  cudaStream_t st = (cudaStream_t)stream;

  ks_ensemble* e = new (std::nothrow) ks_ensemble();
  if (!e) return arg_fail(KS_ERR_INVALID_ARG, "out of host memory");
  e->cfg = *cfg;
  e->cfg.L = nullptr;
  e->cfg.A = nullptr;
  e->M = cfg->n_markets;
  e->N = sz.N;
  e->Lmax = sz.Lmax;
  e->Amax = sz.Amax;
  e->uniform = sz.uniform;
  e->L = sz.L;
  e->A = sz.A;
  e->off = sz.off;
  e->ws = (unsigned char*)workspace;
  e->ws_bytes = ws_bytes;
  cudaError_t ce = cudaGetDevice(&e->device);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device);
  int max_optin = 0;
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, e->device);
  e->max_smem = (size_t)max_optin;
  if (ce != cudaSuccess) {
    delete e;
    return cuda_fail(ce, "device query");
  }

  DevParams& p = e->dp;
  memset(&p, 0, sizeof(p));
  p.M = e->M;
  p.market_base = cfg->market_base;
  p.L_all = sz.L[0];
  p.A_all = sz.A[0];
  p.key0 = (uint32_t)(cfg->seed & 0xffffffffu);
  p.key1 = (uint32_t)(cfg->seed >> 32);
  for (int r = 0; r < 10; ++r) {
    p.rk[2 * r] = p.key0 + (uint32_t)r * PH_WA;
    p.rk[2 * r + 1] = p.key1 + (uint32_t)r * PH_WB;
  }
  p.carry = cfg->carry_book ? 1 : 0;
  p.cancel_thr = cfg->cancel_thresh_q32;
  p.mix0 = cfg->mix_pct[0];
  p.mix01 = cfg->mix_pct[0] + cfg->mix_pct[1];
  p.zi_off = cfg->zi_offset;
  p.zi_qmax = cfg->zi_qmax;
  p.mom_lb = cfg->mom_lookback;
  p.mom_omax = cfg->mom_offset_max;
  p.mr_omax = cfg->mr_offset_max;
  p.rb_qmax = cfg->rb_qmax;
  p.mlp_pct = cfg->mlp_pct;
  p.tie_rule = cfg->tie_rule;
  p.trace_markets = cfg->trace_markets;
  p.trace_steps = cfg->trace_steps;
  p.Lmax = sz.Lmax;
  unsigned char* w = e->ws;
  p.slot = (uint32_t*)(w + lay.slot);
  p.inv = (int32_t*)(w + lay.inv);
  p.cash = (int64_t*)(w + lay.cash);
  p.mi32 = (int32_t*)(w + lay.mi32);
  p.mi64 = (int64_t*)(w + lay.mi64);
  p.agent_off = sz.uniform ? nullptr : (const int64_t*)(w + lay.aoff);
  p.Ls = sz.uniform ? nullptr : (const int32_t*)(w + lay.Ls);
  p.As = sz.uniform ? nullptr : (const int32_t*)(w + lay.As);
  p.trace = (int32_t*)(w + lay.trace);
  p.mlp = (const unsigned char*)cfg->mlp_params;
  p.dec_trace_agents = (uint64_t)sz.off[cfg->trace_markets];
  e->mlp = cfg->mlp_pct > 0;
  p.err = (uint32_t*)(w + lay.ctrl);
  p.step = (const uint64_t*)(w + lay.ctrl + 8);
  e->b_args.ticket = (uint32_t*)(w + lay.ctrl + 16);

  ks_launch l = default_launch(e->Amax, e->M, e->num_sms, e->mlp);
  s = apply_launch(e, &l);
  if (s != KS_OK && sz.uniform) {
    delete e;
    return s;
  }

#define KS_CUDA_E(call)                     \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) {                \
      delete e;                             \
      return cuda_fail(e_, #call);          \
    }                                       \
  } while (0)
  if (!sz.uniform) {
    KS_CUDA_E(cudaMemcpyAsync(w + lay.aoff, sz.off.data(), (size_t)(e->M + 1) * 8, cudaMemcpyHostToDevice, st));
    KS_CUDA_E(cudaMemcpyAsync(w + lay.Ls, sz.L.data(), (size_t)e->M * 4, cudaMemcpyHostToDevice, st));
    KS_CUDA_E(cudaMemcpyAsync(w + lay.As, sz.A.data(), (size_t)e->M * 4, cudaMemcpyHostToDevice, st));
  }
  KS_CUDA_E(cudaMemsetAsync(w + lay.ctrl, 0, 64, st));
  if (lay.ctrl > lay.trace) KS_CUDA_E(cudaMemsetAsync(w + lay.trace, 0, lay.ctrl - lay.trace, st));
  const int grid = (int)std::min<uint32_t>(e->M, 8u * (uint32_t)e->num_sms);
  init_kernel<<<grid, 256, 0, st>>>(p);
  KS_CUDA_E(cudaGetLastError());
  // host copies above read pageable vectors owned by the handle; make sure they are done
  KS_CUDA_E(cudaStreamSynchronize(st));
#undef KS_CUDA_E
  if (!sz.uniform) {
    // uneven ensembles default to the batched kernel with one bucket per (L, A) power-of-two class,
    // in 512-thread CTAs (measured 5-7% faster than 1024-thread CTAs on the 20000- and 32768-market
    // ensembles: a 1024-thread CTA leaves 64 registers per thread)
    const int nt = kDefaultBatchThreads;
    std::vector<ks_bucket> plan = default_plan(e->L, e->A, nt, e->mlp);
    s = build_batch(e, nt, plan.data(), (int)plan.size(), st);
    if (s != KS_OK) {
      delete e;
      return s;
    }
  }
  *out = e;
  return KS_OK;
}

ks_status ks_step_n(ks_ensemble* e, uint32_t n_steps, void* stream) {
  if (!e) return arg_fail(KS_ERR_INVALID_ARG, "ensemble is NULL");
  if (n_steps == 0) return KS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  KS_CUDA(launch_main(e, n_steps, st));
  step_bump_kernel<<<1, 1, 0, st>>>((uint64_t*)e->dp.step, e->b_args.ticket, n_steps);
  KS_CUDA(cudaGetLastError());
  return KS_OK;
}

static ks_status copy_market_field(void* dst, const void* src_base, size_t src_pitch, size_t width, uint32_t M,
                                   cudaStream_t st, bool to_view) {
  if (to_view) {
    KS_CUDA(cudaMemcpy2DAsync(dst, width, src_base, src_pitch, width, M, cudaMemcpyDefault, st));
  } else {
    KS_CUDA(cudaMemcpy2DAsync((void*)src_base, src_pitch, dst, width, width, M, cudaMemcpyDefault, st));
  }
  return KS_OK;
}

static ks_status state_io(ks_ensemble* e, const ks_state_view* v, cudaStream_t st, bool to_view) {
  const DevParams& p = e->dp;
  const size_t N = (size_t)e->N;
  auto lin = [&](void* view, void* dev, size_t bytes) -> ks_status {
    if (!view || bytes == 0) return KS_OK;
    KS_CUDA(cudaMemcpyAsync(to_view ? view : dev, to_view ? dev : view, bytes, cudaMemcpyDefault, st));
    return KS_OK;
  };
  ks_status s;
  if ((s = lin(v->order, p.slot, N * 4)) != KS_OK) return s;
  if ((s = lin(v->inventory, p.inv, N * 4)) != KS_OK) return s;
  if ((s = lin(v->cash, p.cash, N * 8)) != KS_OK) return s;
  const size_t p32 = MI32_STRIDE * 4, p64 = MI64_STRIDE * 8;
  struct F {
    void* view;
    const void* dev;
    size_t pitch, width;
  } fs[] = {
      {v->last_tick, p.mi32 + MI_LAST, p32, 4},
      {v->history, p.mi32 + MI_HIST, p32, 4 * KS_HISTORY},
      {v->fundamental, p.mi32 + MI_FUND, p32, 4},
      {v->trades, p.mi32 + MI_TRADES, p32, 4},
      {v->last_volume, p.mi32 + MI_LASTV, p32, 4},
      {v->sum_price, p.mi64 + MI_SUMP, p64, 8},
      {v->sum_volume, p.mi64 + MI_SUMV, p64, 8},
      {v->trace_hash, p.mi64 + MI_HASH, p64, 8},
  };
  for (auto& f : fs)
    if (f.view && (s = copy_market_field(f.view, f.dev, f.pitch, f.width, e->M, st, to_view)) != KS_OK) return s;
  if ((s = lin(v->step, (void*)p.step, 8)) != KS_OK) return s;
  if ((s = lin(v->trace, p.trace, (size_t)p.trace_markets * p.trace_steps * 2 * 4)) != KS_OK) return s;
  KS_CUDA(cudaStreamSynchronize(st));
  return KS_OK;
}

ks_status ks_read_state(ks_ensemble* e, const ks_state_view* dst, void* stream) {
  if (!e || !dst) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  return state_io(e, dst, (cudaStream_t)stream, true);
}

ks_status ks_write_state(ks_ensemble* e, const ks_state_view* src, void* stream) {
  if (!e || !src) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  return state_io(e, src, (cudaStream_t)stream, false);
}

ks_status ks_error_word(ks_ensemble* e, void* stream, uint32_t* word) {
  if (!e || !word) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  KS_CUDA(cudaMemcpyAsync(word, e->dp.err, 4, cudaMemcpyDeviceToHost, st));
  KS_CUDA(cudaStreamSynchronize(st));
  return KS_OK;
}

ks_status ks_sync(ks_ensemble* e, void* stream, uint32_t timeout_ms) {
  if (!e) return arg_fail(KS_ERR_INVALID_ARG, "ensemble is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ev;
  KS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t ce = cudaEventRecord(ev, st);
  if (ce != cudaSuccess) {
    cudaEventDestroy(ev);
    return cuda_fail(ce, "cudaEventRecord");
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    ce = cudaEventQuery(ev);
    if (ce == cudaSuccess) break;
    if (ce != cudaErrorNotReady) {
      cudaEventDestroy(ev);
      return cuda_fail(ce, "cudaEventQuery");
    }
    if (timeout_ms) {
      const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
      if (ms.count() >= (long long)timeout_ms) {
        cudaEventDestroy(ev);
        return arg_fail(KS_ERR_TIMEOUT, "ks_sync deadline passed before the stream finished");
      }
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  uint32_t word = 0;
  ks_status s = ks_error_word(e, stream, &word);
  if (s != KS_OK) return s;
  if (word) {
    snprintf(g_last_error, sizeof(g_last_error), "device error word 0x%x", word);
    return KS_ERR_DEVICE_FAULT;
  }
  return KS_OK;
}

ks_status ks_set_launch(ks_ensemble* e, const ks_launch* l) {
  if (!e || !l) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  return apply_launch(e, l);
}

ks_status ks_get_launch(const ks_ensemble* e, ks_launch* l) {
  if (!e || !l) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  *l = e->launch;
  return KS_OK;
}

ks_status ks_set_batch_plan(ks_ensemble* e, int32_t cta_threads, const ks_bucket* buckets, int32_t n_buckets,
                            void* stream) {
  if (!e || !buckets) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  return build_batch(e, cta_threads, buckets, n_buckets, (cudaStream_t)stream);
}

ks_status ks_get_batch_info(const ks_ensemble* e, ks_batch_info* info) {
  if (!e || !info) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->batched = e->mode == 1;
  info->cta_threads = e->mode == 1 ? e->b_threads : e->launch.threads;
  info->n_items = e->mode == 1 ? (int32_t)e->b_items.size() : (int32_t)e->M;
  info->n_buckets = e->mode == 1 ? (int32_t)e->b_plan.size() : 1;
  info->grid = e->mode == 1 ? e->b_grid : e->grid;
  info->smem_bytes = (int64_t)(e->mode == 1 ? e->b_smem : e->smem);
  return KS_OK;
}

ks_status ks_set_capture(ks_ensemble* e, const ks_capture* c) {
  if (!e || !c) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  if (c->records && (!c->record_count || c->record_capacity == 0))
    return arg_fail(KS_ERR_INVALID_ARG, "records need record_count and a capacity");
  if ((c->decisions || c->logits) && (e->cfg.trace_markets == 0 || e->cfg.trace_steps == 0))
    return arg_fail(KS_ERR_INVALID_ARG, "decision and logit captures need trace_markets and trace_steps");
  DevParams& p = e->dp;
  p.rec = c->records;
  p.rec_count = c->record_count;
  p.rec_cap = c->records ? c->record_capacity : 0;
  p.rec_agents = c->records ? c->record_agents : 0;
  p.dec_trace = c->decisions;
  p.logit_trace = c->logits;
  p.pol_count = c->policy_count;
  const bool want = e->cfg.mlp_pct > 0 || c->records != nullptr || c->decisions != nullptr || c->logits != nullptr;
  if (want == e->mlp) return KS_OK;
  // switch between the rule-only and the policy-capable kernels, keeping the mode
  e->mlp = want;
  if (e->mode == 1) {
    std::vector<ks_bucket> plan = default_plan(e->L, e->A, kDefaultBatchThreads, e->mlp);
    return build_batch(e, kDefaultBatchThreads, plan.data(), (int)plan.size(), nullptr);
  }
  ks_launch l = default_launch(e->Amax, e->M, e->num_sms, e->mlp);
  return apply_launch(e, &l);
}

ks_status ks_batch_variants(int32_t cta_threads, int32_t* pairs, int32_t capacity, int32_t* count) {
  if (!count) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  int n = 0;
  const int(*tab)[2] = batch_table(cta_threads, &n);
  if (!tab) return arg_fail(KS_ERR_INVALID_ARG, "batched CTA size must be 512 or 1024");
  *count = n;
  if (pairs)
    for (int i = 0; i < n && i < capacity; ++i) {
      pairs[2 * i] = tab[i][0];
      pairs[2 * i + 1] = tab[i][1];
    }
  return KS_OK;
}

ks_status ks_probe_state_io(ks_ensemble* e, void* stream, double* bytes) {
  if (!e || !bytes) return arg_fail(KS_ERR_INVALID_ARG, "NULL argument");
  // zero steps: load every market, rebuild its book, store it back unchanged
  KS_CUDA(launch_main(e, 0u, (cudaStream_t)stream));
  step_bump_kernel<<<1, 1, 0, (cudaStream_t)stream>>>((uint64_t*)e->dp.step, e->b_args.ticket, 0u);
  KS_CUDA(cudaGetLastError());
  *bytes = (double)e->N * 32.0 + (double)e->M * 2.0 * (MI32_STRIDE * 4 + MI64_STRIDE * 8);
  return KS_OK;
}

}  // extern "C"

// Internal accessors for ks_noalloc.cu (no public ABI).
namespace ks {
ks_status internal_batched_schedule(const ks_ensemble* e, const uint32_t** order, const uint4** items,
                                    uint32_t* n_markets, uint32_t* n_items) {
  if (!e) return KS_ERR_INVALID_ARG;
  if (e->mode != 1) return arg_fail(KS_ERR_INVALID_ARG, "the ensemble does not run the batched kernel");
  *order = e->b_order.data();
  *items = e->b_items.data();
  *n_markets = (uint32_t)e->b_order.size();
  *n_items = (uint32_t)e->b_items.size();
  return KS_OK;
}

ks_status internal_launch_batched(ks_ensemble* e, uint32_t n_steps, const BatchArgs& b, cudaStream_t st) {
  cudaError_t ce = e->mlp ? launch_batched_mlp_512(e->dp, n_steps, b, e->b_grid, e->b_smem, st)
                   : e->b_threads == 512 ? launch_batched_512(e->dp, n_steps, b, e->b_grid, e->b_smem, st)
                                         : launch_batched_1024(e->dp, n_steps, b, e->b_grid, e->b_smem, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "batched launch");
  // re-arm the ticket this launch took its items from (b.ticket, not the workspace's)
  step_bump_kernel<<<1, 1, 0, st>>>((uint64_t*)e->dp.step, b.ticket, n_steps);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return cuda_fail(ce, "step counter");
  return KS_OK;
}

int internal_device(const ks_ensemble* e) { return e ? e->device : -1; }

// The initial state of a uniform ensemble described by p (for the CDA ensemble).
cudaError_t internal_init_state(const DevParams& p, int grid, cudaStream_t st) {
  init_kernel<<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}
}  // namespace ks

extern "C" {

ks_status ks_destroy(ks_ensemble* e) {
  delete e;
  return KS_OK;
}

}  // extern "C"
