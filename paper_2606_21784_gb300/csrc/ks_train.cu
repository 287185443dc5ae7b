// ks_train.cu -- behaviour-cloning training of the agent policy: forward,
// loss and backward on the tensor cores, Adam, and export to the BF16 blob
// the step loop reads.
//
// A CTA takes tiles of 64 samples (tile b, b + grid, ...).  Every
// contraction of a tile -- the three forward layers, the two backward
// data products and the three weight-gradient products -- runs as
// mma.sync.m16n8k16 BF16 x BF16 -> FP32 on the tensor cores, with each FP32
// operand passed as a high and a low BF16 part (a = hi + lo; acc += hi*hi +
// hi*lo + lo*hi), so the products keep about 16 mantissa bits and the
// gradient stays within FP32 rounding of the fp64 oracle.  Operands sit in
// shared memory as FP32 and are split when the fragments are built; a
// transposed operand is only a different stride.
//
// Deterministic by construction: every gradient element of a CTA has one
// owner thread that adds the tile products in tile order, the loss of a tile
// is summed in sample order, each CTA writes its partial gradient to the
// caller's workspace, and a second kernel adds the partials in CTA order.
// The grid depends only on the device and n, so the same inputs give the
// same gradient bit for bit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kineticsim.h"
#include "ks_mlp.cuh"

namespace ks {

constexpr int TR_TILE = 64;
constexpr int TR_THREADS = 256;
constexpr int TR_WARPS = TR_THREADS / 32;
constexpr int NP_W1 = MLP_H * MLP_IN, NP_B1 = MLP_H, NP_W2 = MLP_H * MLP_H, NP_B2 = MLP_H;
constexpr int NP_W3 = MLP_OUT * MLP_H, NP_B3 = MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NP_W1, OFF_W2 = OFF_B1 + NP_B1, OFF_B2 = OFF_W2 + NP_W2;
constexpr int OFF_W3 = OFF_B2 + NP_B2, OFF_B3 = OFF_W3 + NP_W3, NPARAM = OFF_B3 + NP_B3;
static_assert(NPARAM == KS_MLP_NPARAM, "parameter count");

constexpr int LDX = MLP_IN + 1;      // padded rows of the [64 x 32] input tile
constexpr int LD = MLP_H + 1;        // padded rows of the [64 x 64] activation tiles
constexpr int NZ = MLP_OUT_PAD;      // output columns padded to 48 (zero beyond 37)
constexpr int LDZ = NZ + 1;
constexpr int PART = NPARAM + 1;     // a CTA's partial: the gradient, then the loss

struct TrainSmem {
  float w[NPARAM];
  float w3p[NZ * MLP_H];             // W3 with rows 37..47 zero
  float g[NPARAM];                   // this CTA's gradient
  float x[TR_TILE][LDX];
  float h1[TR_TILE][LD];
  float h2[TR_TILE][LD];
  float dz[TR_TILE][LDZ];            // logits, then dL/dz
  float d2[TR_TILE][LD];             // dL/da2
  float d1[TR_TILE][LD];             // dL/da1
  float lab_logq[TR_TILE];
  float lsample[TR_TILE];
  int lab_side[TR_TILE];
  int lab_off[TR_TILE];
  float loss;
};

// Normalised inputs of one record (the same reading as the step loop's inputs).
__device__ __forceinline__ float record_feature(const int32_t* r, int k, float invA8, float invA4) {
  if (k < 8) return (float)r[k] * 0.125f;
  if (k == 8) return (float)r[8] * (1.0f / 256.0f);
  if (k == 9) return (float)r[9] * invA8;
  if (k < 18) return (float)r[k] * invA4;
  return 0.0f;
}

// A shared-memory FP32 matrix view: element (r, c) at p[r * rs + c * cs].
struct View {
  const float* p;
  int rs, cs;
  __device__ __forceinline__ float operator()(int r, int c) const { return p[r * rs + c * cs]; }
};

// High and low BF16 parts of two FP32 values, packed as the fragments want
// them (the first value in the low half).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C = A[M x K] * B[K x N] (M a multiple of 16, N of 8, K of 16), one 16 x 8
// output tile per warp at a time; epi(r, c, v) receives every element once,
// from one thread.  Fragment layouts of m16n8k16 (g = lane / 4, t = lane % 4):
// A rows g and g + 8, columns 2t, 2t + 1, 2t + 8, 2t + 9; B rows 2t, 2t + 1,
// 2t + 8, 2t + 9 of column g; C rows g and g + 8, columns 2t and 2t + 1.
template <typename Epi>
__device__ __forceinline__ void tc_gemm(View A, View B, int M, int N, int K, Epi epi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int tn = N / 8, tiles = (M / 16) * tn;
  for (int i = warp; i < tiles; i += TR_WARPS) {
    const int m0 = (i / tn) * 16, n0 = (i % tn) * 8;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int k0 = 0; k0 < K; k0 += 16) {
      uint32_t ah[4], al[4], bh[2], bl[2];
      const int r0 = m0 + g, r1 = r0 + 8, c0 = k0 + 2 * t, c1 = c0 + 8;
      split2(A(r0, c0), A(r0, c0 + 1), ah[0], al[0]);
      split2(A(r1, c0), A(r1, c0 + 1), ah[1], al[1]);
      split2(A(r0, c1), A(r0, c1 + 1), ah[2], al[2]);
      split2(A(r1, c1), A(r1, c1 + 1), ah[3], al[3]);
      const int n = n0 + g;
      split2(B(c0, n), B(c0 + 1, n), bh[0], bl[0]);
      split2(B(c1, n), B(c1 + 1, n), bh[1], bl[1]);
      mma_bf16_16816(acc, al, bh);
      mma_bf16_16816(acc, ah, bl);
      mma_bf16_16816(acc, ah, bh);
    }
    epi(m0 + g, n0 + 2 * t, acc[0]);
    epi(m0 + g, n0 + 2 * t + 1, acc[1]);
    epi(m0 + g + 8, n0 + 2 * t, acc[2]);
    epi(m0 + g + 8, n0 + 2 * t + 1, acc[3]);
  }
}

__global__ void __launch_bounds__(TR_THREADS) bc_grad_kernel(const float* __restrict__ params,
                                                             const int32_t* __restrict__ rec, int64_t n, int A,
                                                             float* __restrict__ part, float scale) {
  extern __shared__ __align__(16) unsigned char raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(raw);
  const int tid = threadIdx.x;
  for (int i = tid; i < NPARAM; i += TR_THREADS) {
    S.w[i] = params[i];
    S.g[i] = 0.0f;
  }
  for (int i = tid; i < NZ * MLP_H; i += TR_THREADS) S.w3p[i] = i < NP_W3 ? params[OFF_W3 + i] : 0.0f;
  if (tid == 0) S.loss = 0.0f;
  const float invA8 = 1.0f / (8.0f * (float)max(A, 1));
  const float invA4 = 1.0f / (4.0f * (float)max(A, 1));
  float* const gw = S.g;
  const float* b1 = S.w + OFF_B1;
  const float* b2 = S.w + OFF_B2;
  const float* b3 = S.w + OFF_B3;
  // operand views (row, column) -> element
  const View vX{&S.x[0][0], LDX, 1}, vH1{&S.h1[0][0], LD, 1}, vH2{&S.h2[0][0], LD, 1};
  const View vDZ{&S.dz[0][0], LDZ, 1}, vD2{&S.d2[0][0], LD, 1};
  const View vXt{&S.x[0][0], 1, LDX}, vH1t{&S.h1[0][0], 1, LD}, vH2t{&S.h2[0][0], 1, LD};
  const View vDZt{&S.dz[0][0], 1, LDZ}, vD2t{&S.d2[0][0], 1, LD}, vD1t{&S.d1[0][0], 1, LD};
  const View vW1t{S.w + OFF_W1, 1, MLP_IN};   // (k, n) = W1[n][k]
  const View vW2t{S.w + OFF_W2, 1, MLP_H};    // (k, n) = W2[n][k]
  const View vW2{S.w + OFF_W2, MLP_H, 1};     // (k, n) = W2[k][n]
  const View vW3t{S.w3p, 1, MLP_H};           // (k, n) = W3[n][k]
  const View vW3{S.w3p, MLP_H, 1};            // (k, n) = W3[k][n]
  const int64_t ntiles = (n + TR_TILE - 1) / TR_TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * TR_TILE;
    const int cnt = (int)min((int64_t)TR_TILE, n - base);
    __syncthreads();
    // inputs and labels (rows beyond the tail: zero inputs, no loss)
    for (int i = tid; i < TR_TILE * MLP_IN; i += TR_THREADS) {
      const int r = i / MLP_IN, k = i % MLP_IN;
      S.x[r][k] = r < cnt ? record_feature(rec + (base + r) * KS_RECORD_WORDS, k, invA8, invA4) : 0.0f;
    }
    if (tid < TR_TILE) {
      const int32_t* rr = rec + (base + min(tid, cnt - 1)) * KS_RECORD_WORDS;
      S.lab_side[tid] = rr[18];
      S.lab_off[tid] = rr[19];
      S.lab_logq[tid] = logf((float)max(rr[20], 1));
    }
    __syncthreads();
    // forward: h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), z = h2 W3^T + b3
    tc_gemm(vX, vW1t, TR_TILE, MLP_H, MLP_IN, [&](int r, int c, float v) { S.h1[r][c] = fmaxf(v + b1[c], 0.0f); });
    __syncthreads();
    tc_gemm(vH1, vW2t, TR_TILE, MLP_H, MLP_H, [&](int r, int c, float v) { S.h2[r][c] = fmaxf(v + b2[c], 0.0f); });
    __syncthreads();
    tc_gemm(vH2, vW3t, TR_TILE, NZ, MLP_H,
            [&](int r, int c, float v) { S.dz[r][c] = c < MLP_OUT ? v + b3[c] : 0.0f; });
    __syncthreads();
    // loss and dL/dz per sample (softmax cross-entropy x2, squared error)
    if (tid < TR_TILE) {
      float* z = S.dz[tid];
      const bool ok = tid < cnt;
      float l = 0.0f;
      {
        float mx = z[0];
        for (int i = 1; i < MLP_NSIDE; ++i) mx = fmaxf(mx, z[i]);
        float se = 0.0f;
        for (int i = 0; i < MLP_NSIDE; ++i) se += expf(z[i] - mx);
        const int y = S.lab_side[tid];
        l -= z[y] - mx - logf(se);
        for (int i = 0; i < MLP_NSIDE; ++i) z[i] = expf(z[i] - mx) / se - (i == y ? 1.0f : 0.0f);
      }
      {
        float* zo = z + MLP_NSIDE;
        float mx = zo[0];
        for (int i = 1; i < MLP_NOFF; ++i) mx = fmaxf(mx, zo[i]);
        float se = 0.0f;
        for (int i = 0; i < MLP_NOFF; ++i) se += expf(zo[i] - mx);
        const int y = S.lab_off[tid];
        l -= zo[y] - mx - logf(se);
        for (int i = 0; i < MLP_NOFF; ++i) zo[i] = expf(zo[i] - mx) / se - (i == y ? 1.0f : 0.0f);
      }
      const float e = z[MLP_OUT - 1] - S.lab_logq[tid];
      l += e * e;
      z[MLP_OUT - 1] = 2.0f * e;
      for (int i = 0; i < MLP_OUT; ++i) z[i] = ok ? z[i] * scale : 0.0f;
      S.lsample[tid] = ok ? l * scale : 0.0f;
    }
    __syncthreads();
    if (tid == 0) {
      float s = 0.0f;
      for (int r = 0; r < TR_TILE; ++r) s += S.lsample[r];
      S.loss += s;
    }
    // d2 = (dz W3) * [h2 > 0];  gW3 += dz^T h2;  gb3 += column sums of dz
    tc_gemm(vDZ, vW3, TR_TILE, MLP_H, NZ,
            [&](int r, int c, float v) { S.d2[r][c] = S.h2[r][c] > 0.0f ? v : 0.0f; });
    tc_gemm(vDZt, vH2, NZ, MLP_H, TR_TILE, [&](int r, int c, float v) {
      if (r < MLP_OUT) gw[OFF_W3 + r * MLP_H + c] += v;
    });
    if (tid < MLP_OUT) {
      float a = 0.0f;
      for (int r = 0; r < TR_TILE; ++r) a += S.dz[r][tid];
      gw[OFF_B3 + tid] += a;
    }
    __syncthreads();
    // d1 = (d2 W2) * [h1 > 0];  gW2 += d2^T h1;  gb2 += column sums of d2
    tc_gemm(vD2, vW2, TR_TILE, MLP_H, MLP_H,
            [&](int r, int c, float v) { S.d1[r][c] = S.h1[r][c] > 0.0f ? v : 0.0f; });
    tc_gemm(vD2t, vH1, MLP_H, MLP_H, TR_TILE, [&](int r, int c, float v) { gw[OFF_W2 + r * MLP_H + c] += v; });
    if (tid < MLP_H) {
      float a = 0.0f;
      for (int r = 0; r < TR_TILE; ++r) a += S.d2[r][tid];
      gw[OFF_B2 + tid] += a;
    }
    __syncthreads();
    // gW1 += d1^T x;  gb1 += column sums of d1
    tc_gemm(vD1t, vX, MLP_H, MLP_IN, TR_TILE, [&](int r, int c, float v) { gw[OFF_W1 + r * MLP_IN + c] += v; });
    if (tid < MLP_H) {
      float a = 0.0f;
      for (int r = 0; r < TR_TILE; ++r) a += S.d1[r][tid];
      gw[OFF_B1 + tid] += a;
    }
  }
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * PART;
  for (int i = tid; i < NPARAM; i += TR_THREADS) out[i] = S.g[i];
  if (tid == 0) out[NPARAM] = S.loss;
  (void)vH1t;
  (void)vH2t;
  (void)vXt;
}

// grad[i] += sum over CTAs c = 0, 1, ... of part[c][i] (in that order); the
// loss the same way.
__global__ void bc_reduce_kernel(const float* __restrict__ part, int nblk, float* __restrict__ grad,
                                 float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= PART) return;
  float s = 0.0f;
  for (int c = 0; c < nblk; ++c) s += part[(size_t)c * PART + i];
  if (i < NPARAM)
    grad[i] += s;
  else
    loss[0] += s;
}

// Adam with bias correction (Kingma and Ba, 2015); zeroes the gradient.
__global__ void adam_kernel(float* w, float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  g[i] = 0.0f;
}

// FP32 parameter vector -> the step loop's blob (BF16 weights, FP32 biases).
__global__ void export_kernel(const float* w, unsigned char* blob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  __nv_bfloat16* W1 = reinterpret_cast<__nv_bfloat16*>(blob + MLP_OFF_W1);
  __nv_bfloat16* W2 = reinterpret_cast<__nv_bfloat16*>(blob + MLP_OFF_W2);
  __nv_bfloat16* W3 = reinterpret_cast<__nv_bfloat16*>(blob + MLP_OFF_W3);
  float* B1 = reinterpret_cast<float*>(blob + MLP_OFF_B1);
  float* B2 = reinterpret_cast<float*>(blob + MLP_OFF_B2);
  float* B3 = reinterpret_cast<float*>(blob + MLP_OFF_B3);
  if (i < NP_W1) W1[i] = __float2bfloat16_rn(w[OFF_W1 + i]);
  if (i < NP_W2) W2[i] = __float2bfloat16_rn(w[OFF_W2 + i]);
  if (i < NP_W3) W3[i] = __float2bfloat16_rn(w[OFF_W3 + i]);
  if (i < NP_B1) B1[i] = w[OFF_B1 + i];
  if (i < NP_B2) B2[i] = w[OFF_B2 + i];
  if (i < NP_B3) B3[i] = w[OFF_B3 + i];
}

}  // namespace ks

namespace ks {
// CTAs of a gradient launch over n samples on the current device.
static int bc_grid(int64_t n) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess)
    return -1;
  const int64_t ntiles = (n + TR_TILE - 1) / TR_TILE;
  return (int)(ntiles < (int64_t)sms ? ntiles : (int64_t)sms);
}
}  // namespace ks

extern "C" ks_status ks_bc_workspace_size(int64_t n, size_t* bytes) {
  if (!bytes || n < 0) return KS_ERR_INVALID_ARG;
  const int grid = n > 0 ? ks::bc_grid(n) : 0;
  if (grid < 0) return KS_ERR_CUDA;
  *bytes = (size_t)grid * ks::PART * sizeof(float);
  return KS_OK;
}

extern "C" ks_status ks_bc_grad(const float* params, const int32_t* records, int64_t n, int32_t A, float* grad,
                                float* loss, float scale, void* workspace, size_t ws_bytes, void* stream) {
  if (!params || !grad || !loss || n < 0 || (n > 0 && !records) || A < 1) return KS_ERR_INVALID_ARG;
  if (n == 0) return KS_OK;
  const int grid = ks::bc_grid(n);
  if (grid < 0) return KS_ERR_CUDA;
  if (!workspace || ws_bytes < (size_t)grid * ks::PART * sizeof(float)) return KS_ERR_WORKSPACE_TOO_SMALL;
  const size_t smem = sizeof(ks::TrainSmem);
  if (cudaFuncSetAttribute(ks::bc_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return KS_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  float* part = (float*)workspace;
  ks::bc_grad_kernel<<<grid, ks::TR_THREADS, smem, st>>>(params, records, n, A, part, scale);
  if (cudaGetLastError() != cudaSuccess) return KS_ERR_CUDA;
  ks::bc_reduce_kernel<<<(ks::PART + 255) / 256, 256, 0, st>>>(part, grid, grad, loss);
  return cudaGetLastError() == cudaSuccess ? KS_OK : KS_ERR_CUDA;
}

extern "C" ks_status ks_adam_step(float* params, float* grad, float* m, float* v, int32_t step, float lr, float beta1,
                                  float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || step < 1) return KS_ERR_INVALID_ARG;
  const float c1 = 1.0f - powf(beta1, (float)step);
  const float c2 = 1.0f - powf(beta2, (float)step);
  const int n = ks::NPARAM;
  ks::adam_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, lr, beta1, beta2, eps, c1,
                                                                       c2);
  return cudaGetLastError() == cudaSuccess ? KS_OK : KS_ERR_CUDA;
}

extern "C" ks_status ks_mlp_export(const float* params, void* blob, void* stream) {
  if (!params || !blob || ((uintptr_t)blob & 15u) != 0) return KS_ERR_INVALID_ARG;
  ks::export_kernel<<<(ks::NP_W2 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, (unsigned char*)blob);
  return cudaGetLastError() == cudaSuccess ? KS_OK : KS_ERR_CUDA;
}
