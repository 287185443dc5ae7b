// ks_mlp.cuh -- the agent policy network on sm_103a tensor cores.
//
// Policy 32 -> 64 -> 64 -> 37 (3 side logits, 33 tick-offset logits, 1
// log-quantity), ReLU hidden layers, BF16 weights, FP32 accumulation.
// Layer 1 runs in FP32 on the CUDA cores (inside the step loop it is a
// rank-1 update per agent: only the inventory input differs between the
// agents of a market).  Layers 2 and 3 are dense 64-wide contractions on the
// tensor cores: one warpgroup (128 threads) evaluates a tile of 128 agents,
// thread r owning row r; each layer is a chain of M=128, K=16 tcgen05.mma
// (kind::f16, BF16 x BF16 -> FP32 in tensor memory) committed to an
// mbarrier.  The weights are K-major no-swizzle operands in shared memory;
// the activations are the A operand in tensor memory: thread r writes its
// row into TMEM lane r with tcgen05.st, so a tile needs no shared-memory
// activation buffer and every warpgroup of a CTA can run tiles.  The
// activation operand is passed as a high and a low BF16 part (a = hi + lo,
// two MMAs per K chunk into the same accumulator), so the only rounding left
// in the contraction is that of the BF16 weights themselves.  The epilogue
// reads the accumulator rows with tcgen05.ld and adds the bias.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "kineticsim.h"
#include "ks_internal.h"
#include "ks_tc.cuh"

namespace ks {

constexpr int MLP_IN = 32;
constexpr int MLP_H = 64;
constexpr int MLP_OUT = 37;
constexpr int MLP_OUT_PAD = 48;
constexpr int MLP_NSIDE = 3;
constexpr int MLP_NOFF = 33;
constexpr int MLP_OFF_MAX = 16;

// Parameter blob (see kineticsim.h): row-major (out, in) BF16 weights, FP32 biases.
constexpr uint32_t MLP_OFF_W1 = 0;
constexpr uint32_t MLP_OFF_W2 = MLP_OFF_W1 + 2 * MLP_H * MLP_IN;
constexpr uint32_t MLP_OFF_W3 = MLP_OFF_W2 + 2 * MLP_H * MLP_H;
constexpr uint32_t MLP_OFF_B1 = MLP_OFF_W3 + 2 * MLP_OUT * MLP_H;
constexpr uint32_t MLP_OFF_B2 = MLP_OFF_B1 + 4 * MLP_H;
constexpr uint32_t MLP_OFF_B3 = MLP_OFF_B2 + 4 * MLP_H;
constexpr uint32_t MLP_PARAM_BYTES_RAW = MLP_OFF_B3 + 4 * MLP_OUT;
static_assert(MLP_PARAM_BYTES_RAW <= KS_MLP_PARAM_BYTES, "parameter blob size");

// Shared memory of the weights (per CTA): W1 as FP32 row-major for the CUDA
// cores, W2 and W3 as BF16 tensor-core operands.
constexpr uint32_t MLP_SM_W1 = 0;                               // f32 [64][32]
constexpr uint32_t MLP_SM_W2 = MLP_SM_W1 + 4 * MLP_H * MLP_IN;    // bf16 [64 x 64] operand layout
constexpr uint32_t MLP_SM_W3 = MLP_SM_W2 + 2 * MLP_H * MLP_H;     // bf16 [48 x 64], rows 37..47 zero
constexpr uint32_t MLP_SM_B = MLP_SM_W3 + 2 * MLP_OUT_PAD * MLP_H;  // f32 b1[64] b2[64] b3[48]
// f32 [64]: column 8 of W1 (the inventory input) stored contiguously for the step loop's layer 1
constexpr uint32_t MLP_SM_W1INV = MLP_SM_B + 4 * (MLP_H + MLP_H + MLP_OUT_PAD);
constexpr uint32_t MLP_SM_BYTES = MLP_SM_W1INV + 4 * MLP_H;
// TMEM columns of a tile warpgroup: the FP32 accumulator (64 columns), then
// the hidden activations as the A operand, high part and low part (64 BF16
// per row = 32 columns each).  At most four tile warpgroups fit an SM's 512.
constexpr uint32_t MLP_TMEM_ACC = 0;
constexpr uint32_t MLP_TMEM_AHI = 64;
constexpr uint32_t MLP_TMEM_ALO = 96;
constexpr uint32_t MLP_TMEM_COLS = 128;  // per tile warpgroup
constexpr int MLP_MAX_TILE_WGS = 4;
constexpr uint32_t MLP_WAIT_LIMIT = 1u << 22;

// Loads the blob into the operand layout; all threads of the CTA take part.
__device__ __forceinline__ void mlp_load_weights(const unsigned char* blob, unsigned char* sw, int tid, int nthr) {
  const __nv_bfloat16* W1 = reinterpret_cast<const __nv_bfloat16*>(blob + MLP_OFF_W1);
  const __nv_bfloat16* W2 = reinterpret_cast<const __nv_bfloat16*>(blob + MLP_OFF_W2);
  const __nv_bfloat16* W3 = reinterpret_cast<const __nv_bfloat16*>(blob + MLP_OFF_W3);
  float* w1f = reinterpret_cast<float*>(sw + MLP_SM_W1);
  for (int i = tid; i < MLP_H * MLP_IN; i += nthr) w1f[i] = __bfloat162float(W1[i]);
  for (int i = tid; i < MLP_H * MLP_H; i += nthr) {
    const int r = i / MLP_H, k = i % MLP_H;
    *reinterpret_cast<__nv_bfloat16*>(sw + MLP_SM_W2 + cm_offset(r, k, MLP_H)) = W2[i];
  }
  for (int i = tid; i < MLP_OUT_PAD * MLP_H; i += nthr) {
    const int r = i / MLP_H, k = i % MLP_H;
    *reinterpret_cast<__nv_bfloat16*>(sw + MLP_SM_W3 + cm_offset(r, k, MLP_H)) =
        r < MLP_OUT ? W3[r * MLP_H + k] : __float2bfloat16(0.0f);
  }
  const float* b1 = reinterpret_cast<const float*>(blob + MLP_OFF_B1);
  const float* b2 = reinterpret_cast<const float*>(blob + MLP_OFF_B2);
  const float* b3 = reinterpret_cast<const float*>(blob + MLP_OFF_B3);
  float* sb = reinterpret_cast<float*>(sw + MLP_SM_B);
  for (int i = tid; i < MLP_H + MLP_H + MLP_OUT_PAD; i += nthr) {
    float v;
    if (i < MLP_H) v = b1[i];
    else if (i < 2 * MLP_H) v = b2[i - MLP_H];
    else v = (i - 2 * MLP_H) < MLP_OUT ? b3[i - 2 * MLP_H] : 0.0f;
    sb[i] = v;
  }
  float* w1i = reinterpret_cast<float*>(sw + MLP_SM_W1INV);
  for (int i = tid; i < MLP_H; i += nthr) w1i[i] = __bfloat162float(W1[i * MLP_IN + 8]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// Barrier of `count` threads that also ORs a predicate over them.
__device__ __forceinline__ bool named_sync_or(int id, int count, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.b32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return out != 0;
}

// State of one warpgroup's tile pipeline.
struct MlpWG {
  uint64_t* bar;       // mbarrier (count 1)
  uint32_t tmem;       // TMEM address of this warpgroup's MLP_TMEM_COLS columns
  int bar_id;          // named barrier of the 128 threads
  uint32_t phase;      // parity of the next mbarrier completion
  bool abort;          // a bounded wait gave up: no further MMAs
  int wg;              // this warpgroup's index in its market group
  int nwg;             // warpgroups of the group that evaluate policy tiles (those with wg < nwg)
};

// Issues one layer: for each 16-wide K chunk (8 TMEM columns of the
// activations), acc += hi * W and acc += lo * W; then commits the chain to
// the warpgroup's mbarrier.
__device__ __forceinline__ void mlp_issue(const MlpWG& g, uint32_t b_addr, int N) {
  tc_fence_after();
  const uint32_t idesc = idesc_bf16_f32(128, N);
  const uint32_t sbo = (uint32_t)MLP_H * 16;
  for (int kk = 0; kk < MLP_H / 16; ++kk) {
    const uint64_t bd = smem_desc(b_addr + 256u * kk, 128u, sbo);
    mma_bf16_ts(g.tmem + MLP_TMEM_ACC, g.tmem + MLP_TMEM_AHI + 8u * kk, bd, idesc, kk > 0);
    mma_bf16_ts(g.tmem + MLP_TMEM_ACC, g.tmem + MLP_TMEM_ALO + 8u * kk, bd, idesc, true);
  }
  mma_commit(g.bar);
}

// The bounded part of a layer wait: the issuing thread polls the mbarrier
// (at most MLP_WAIT_LIMIT times), the others wait at the warpgroup's named
// barrier, which also spreads a timeout.  On the first timeout the warpgroup
// records ERR_MLP_WAIT and stops waiting (and issuing) for good.
__device__ __forceinline__ void mlp_wait_bounded(MlpWG& g, uint32_t* err) {
  bool ok = true;
  if ((threadIdx.x & 127) == 0) ok = g.abort ? false : mbar_wait_bounded(g.bar, g.phase, MLP_WAIT_LIMIT);
  const bool any_fail = named_sync_or(g.bar_id, 128, !ok) || g.abort;
  if (any_fail && !g.abort) {
    g.abort = true;
    if ((threadIdx.x & 127) == 0) atomicOr(err, ERR_MLP_WAIT);
  }
  g.phase ^= 1u;
}

// Waits for the layer's MMAs.
__device__ __forceinline__ void mlp_wait(MlpWG& g, uint32_t* err) {
  mlp_wait_bounded(g, err);
  tc_fence_after();
}

// Reads `ncols` accumulator columns of this thread's row (multiple of 16).
__device__ __forceinline__ void mlp_read(const MlpWG& g, int ncols, float* v) {
  const uint32_t lane_base = (uint32_t)((threadIdx.x >> 5) & 3) * 32u;
  for (int c = 0; c < ncols; c += 16) tmem_ld16(g.tmem + (lane_base << 16) + (uint32_t)c, v + c);
  tmem_wait_ld();
}

// Writes activations [8 kc, 8 kc + 8) of this thread's row into the A
// operand in TMEM as high and low BF16 parts: hi = bf16(h), lo = bf16(h - hi),
// two elements per column (columns 4 kc .. 4 kc + 3 of each part).
__device__ __forceinline__ void mlp_tstore8(const MlpWG& g, int kc, const float* h) {
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float a = h[2 * j], b = h[2 * j + 1];
    hi[j] = pack_bf16x2(a, b);
    const float ah = __uint_as_float(hi[j] << 16), bh = __uint_as_float(hi[j] & 0xFFFF0000u);
    lo[j] = pack_bf16x2(a - ah, b - bh);
  }
  const uint32_t lane = ((threadIdx.x >> 5) & 3u) * 32u;
  const uint32_t t = g.tmem + (lane << 16) + 4u * (uint32_t)kc;
  tmem_st4(t + MLP_TMEM_AHI, hi[0], hi[1], hi[2], hi[3]);
  tmem_st4(t + MLP_TMEM_ALO, lo[0], lo[1], lo[2], lo[3]);
}

// The warpgroup's activation stores are complete and visible to the MMA the
// issuing thread starts next.
__device__ __forceinline__ void mlp_operand_ready(const MlpWG& g) {
  tmem_wait_st();
  tc_fence_before();
  named_sync(g.bar_id, 128);
}

// Layers 2 and 3 of one 128-row tile.  h1: this thread's 64 first-layer
// activations (after ReLU); z: its 37 logits.  All 128 threads of the
// warpgroup call it together.
__device__ __forceinline__ void mlp_tile_forward(MlpWG& g, const unsigned char* sw, const float* h1, float* z,
                                                 uint32_t* err) {
  const int r = (int)(threadIdx.x & 127);
  const float* sb = reinterpret_cast<const float*>(sw + MLP_SM_B);
  const uint32_t w_addr = smem_u32(sw);
  float acc[MLP_H];
#pragma unroll
  for (int kc = 0; kc < MLP_H / 8; ++kc) mlp_tstore8(g, kc, h1 + 8 * kc);
  mlp_operand_ready(g);
  if (r == 0 && !g.abort) mlp_issue(g, w_addr + MLP_SM_W2, MLP_H);
  mlp_wait(g, err);
  mlp_read(g, MLP_H, acc);
#pragma unroll
  for (int i = 0; i < MLP_H; ++i) acc[i] = fmaxf(acc[i] + sb[MLP_H + i], 0.0f);
#pragma unroll
  for (int kc = 0; kc < MLP_H / 8; ++kc) mlp_tstore8(g, kc, acc + 8 * kc);  // layer 2 read its operand already
  mlp_operand_ready(g);
  if (r == 0 && !g.abort) mlp_issue(g, w_addr + MLP_SM_W3, MLP_OUT_PAD);
  mlp_wait(g, err);
  mlp_read(g, MLP_OUT_PAD, acc);
#pragma unroll
  for (int i = 0; i < MLP_OUT; ++i) z[i] = g.abort ? 0.0f : acc[i] + sb[2 * MLP_H + i];
  tc_fence_before();
}

// First layer in FP32 from a full input row (W1 row-major in shared memory).
__device__ __forceinline__ void mlp_layer1(const unsigned char* sw, const float* x, float* h1) {
  const float* w1 = reinterpret_cast<const float*>(sw + MLP_SM_W1);
  const float* b1 = reinterpret_cast<const float*>(sw + MLP_SM_B);
#pragma unroll 4
  for (int i = 0; i < MLP_H; ++i) {
    float a = b1[i];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) a = fmaf(w1[i * MLP_IN + k], x[k], a);
    h1[i] = fmaxf(a, 0.0f);
  }
}

// ---------------------------------------------------------------------------------------------
// CTA-level resources of the policy path: the weights (loaded once per
// launch), one mbarrier per market group and the CTA's TMEM allocation
// (64 columns per group).  Each group's activation buffer sits after its
// market shared memory.
// ---------------------------------------------------------------------------------------------
constexpr int MLP_MAX_GROUPS = 16;
__host__ __device__ constexpr uint32_t mlp_cta_bytes() {
  return ((MLP_SM_BYTES + 127u) & ~127u) + 8u * MLP_MAX_GROUPS + 16u;
}

struct MlpCta {
  unsigned char* sw;
  uint64_t* bars;
  uint32_t* tslot;
  uint32_t cols;
};

__device__ __forceinline__ MlpCta mlp_cta_carve(unsigned char* raw, uint32_t cols) {
  MlpCta c;
  c.sw = raw;
  c.bars = reinterpret_cast<uint64_t*>(raw + ((MLP_SM_BYTES + 127u) & ~127u));
  c.tslot = reinterpret_cast<uint32_t*>(c.bars + MLP_MAX_GROUPS);
  c.cols = cols;
  return c;
}

// Whole CTA: TMEM allocation (warp 0), mbarriers (thread 0), weights.
__device__ __forceinline__ void mlp_cta_setup(const MlpCta& c, const unsigned char* blob) {
  if (threadIdx.x < 32) {
    tmem_alloc(c.tslot, c.cols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < MLP_MAX_GROUPS; ++i) mbar_init(&c.bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (blob) mlp_load_weights(blob, c.sw, (int)threadIdx.x, (int)blockDim.x);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Whole CTA: frees the TMEM columns once every group is done.
__device__ __forceinline__ void mlp_cta_teardown(const MlpCta& c) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(*c.tslot, c.cols);
  }
}

// ---------------------------------------------------------------------------------------------
// Decision of an MLP agent from its logits and its Philox stream-3 words:
// inverse-CDF draws of side (w0) and tick offset (w1) from the softmax of
// their heads, quantity clamp(round(exp(z[36])), 1, qmax).
// ---------------------------------------------------------------------------------------------
// Largest of z[0, N) as a pairwise tree (max is exact in any order).
template <int N>
__device__ __forceinline__ float max_tree(const float* z) {
  if constexpr (N == 1) {
    return z[0];
  } else {
    return fmaxf(max_tree<N / 2>(z), max_tree<N - N / 2>(z + N / 2));
  }
}

template <int N>
__device__ __forceinline__ int mlp_sample(const float* z, uint32_t w) {
  const float mx = max_tree<N>(z);
  // running sums c_i of exp(z - max); the total is c_{N-1}
  float c[N];
  float run = 0.0f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    run += __expf(z[i] - mx);
    c[i] = run;
  }
  const float u = (float)w * 2.3283064365386963e-10f * run;  // u * sum, compared with the running sums
  // first i with u < c_i (N - 1 if none): c is non-decreasing, so it is the
  // number of i < N - 1 with c_i <= u
  int pick = 0;
#pragma unroll
  for (int i = 0; i < N - 1; ++i) pick += (c[i] <= u) ? 1 : 0;
  return pick;
}


// Step-loop policy tile: layer 1 is c + W1[:, 8] * x_inv (c: the 64
// pre-activations shared by the market's agents, x_inv: this row's inventory
// input), layers 2-3 on the tensor cores, 16 accumulator columns at a time.
// Returns the 37 logits of this thread's row.
__device__ __forceinline__ void mlp_tile_logits(MlpWG& g, const unsigned char* sw, const float* cvec, float x_inv,
                                                float* z, uint32_t* err) {
  const int r = (int)(threadIdx.x & 127);
  const float4* w1i = reinterpret_cast<const float4*>(sw + MLP_SM_W1INV);
  const float4* cv = reinterpret_cast<const float4*>(cvec);
  const float* sb = reinterpret_cast<const float*>(sw + MLP_SM_B);
  const uint32_t w_addr = smem_u32(sw);
  const uint32_t lane_base = (uint32_t)((threadIdx.x >> 5) & 3) * 32u;
#pragma unroll 1
  for (int kc = 0; kc < MLP_H / 8; ++kc) {
    const float4 wa = w1i[2 * kc], wb = w1i[2 * kc + 1], ca = cv[2 * kc], cb = cv[2 * kc + 1];
    const float h[8] = {fmaxf(fmaf(wa.x, x_inv, ca.x), 0.0f), fmaxf(fmaf(wa.y, x_inv, ca.y), 0.0f),
                        fmaxf(fmaf(wa.z, x_inv, ca.z), 0.0f), fmaxf(fmaf(wa.w, x_inv, ca.w), 0.0f),
                        fmaxf(fmaf(wb.x, x_inv, cb.x), 0.0f), fmaxf(fmaf(wb.y, x_inv, cb.y), 0.0f),
                        fmaxf(fmaf(wb.z, x_inv, cb.z), 0.0f), fmaxf(fmaf(wb.w, x_inv, cb.w), 0.0f)};
    mlp_tstore8(g, kc, h);
  }
  mlp_operand_ready(g);
  if (r == 0 && !g.abort) mlp_issue(g, w_addr + MLP_SM_W2, MLP_H);
  mlp_wait(g, err);
#pragma unroll 1
  for (int c = 0; c < MLP_H / 16; ++c) {
    float v[16];
    tmem_ld16(g.tmem + (lane_base << 16) + MLP_TMEM_ACC + (uint32_t)(16 * c), v);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + sb[MLP_H + 16 * c + j], 0.0f);
    mlp_tstore8(g, 2 * c, v);  // layer 2 has read its operand: overwrite it with layer 3's
    mlp_tstore8(g, 2 * c + 1, v + 8);
  }
  mlp_operand_ready(g);
  if (r == 0 && !g.abort) mlp_issue(g, w_addr + MLP_SM_W3, MLP_OUT_PAD);
  mlp_wait(g, err);
#pragma unroll
  for (int c = 0; c < MLP_OUT_PAD / 16; ++c) {
    float v[16];
    tmem_ld16(g.tmem + (lane_base << 16) + MLP_TMEM_ACC + (uint32_t)(16 * c), v);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (16 * c + j < MLP_OUT) z[16 * c + j] = g.abort ? 0.0f : v[j] + sb[2 * MLP_H + 16 * c + j];
  }
  tc_fence_before();
}

// Order word of a policy decision (qty | side << 8 | tick << 9), or
// KS_DECISION_PASS.  w: the agent's Philox stream-3 block for the step.
__device__ __forceinline__ uint32_t mlp_decision(const float* z, uint4 w, int last, int L, int qmax) {
  const int side = mlp_sample<MLP_NSIDE>(z, w.x);
  if (side == 2) return KS_DECISION_PASS;
  const int oi = mlp_sample<MLP_NOFF>(z + MLP_NSIDE, w.y);
  float q = floorf(expf(z[MLP_OUT - 1]) + 0.5f);
  q = (q >= 1.0f) ? q : 1.0f;  // also maps NaN to 1
  q = fminf(q, (float)qmax);
  const int k = oi - MLP_OFF_MAX;  // ticks toward the opposite side: up for a buy, down for a sell
  const int tick = min(max(last + (side ? -k : k), 0), L - 1);
  return (uint32_t)q | ((uint32_t)side << 8) | ((uint32_t)tick << 9);
}

}  // namespace ks
