// ks_train.cu -- behaviour-cloning training of the agent policy: forward,
// loss, backward (FP32, CUDA cores), Adam, and export to the BF16 blob the
// step loop reads.
//
// The policy is tiny (8677 parameters) and a minibatch is a few thousand
// samples, so each contraction is a few hundred thousand multiply-adds: the
// kernels keep the weights and one 64-sample tile's activations in shared
// memory, use all 256 threads of a CTA on every layer, and add each CTA's
// partial gradient into the global gradient with one atomic per parameter.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kineticsim.h"
#include "ks_mlp.cuh"

namespace ks {

constexpr int TR_TILE = 64;
constexpr int TR_THREADS = 256;
constexpr int NP_W1 = MLP_H * MLP_IN, NP_B1 = MLP_H, NP_W2 = MLP_H * MLP_H, NP_B2 = MLP_H;
constexpr int NP_W3 = MLP_OUT * MLP_H, NP_B3 = MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NP_W1, OFF_W2 = OFF_B1 + NP_B1, OFF_B2 = OFF_W2 + NP_W2;
constexpr int OFF_W3 = OFF_B2 + NP_B2, OFF_B3 = OFF_W3 + NP_W3, NPARAM = OFF_B3 + NP_B3;
static_assert(NPARAM == KS_MLP_NPARAM, "parameter count");

constexpr int LD = MLP_H + 1;  // padded row of the [64 x 64] activation tiles
constexpr int LDZ = MLP_OUT + 1;

struct TrainSmem {
  float w[NPARAM];
  float g[NPARAM];                 // this CTA's partial gradient
  float x[TR_TILE][MLP_IN + 1];
  float h1[TR_TILE][LD];
  float h2[TR_TILE][LD];
  float dz[TR_TILE][LDZ];
  float d2[TR_TILE][LD];           // dL/da2
  float d1[TR_TILE][LD];           // dL/da1
  float lab_logq[TR_TILE];
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

__global__ void __launch_bounds__(TR_THREADS) bc_grad_kernel(const float* __restrict__ params,
                                                             const int32_t* __restrict__ rec, int64_t n, int A,
                                                             float* __restrict__ grad, float* __restrict__ loss_out,
                                                             float scale) {
  extern __shared__ __align__(16) unsigned char raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(raw);
  const int tid = threadIdx.x;
  for (int i = tid; i < NPARAM; i += TR_THREADS) {
    S.w[i] = params[i];
    S.g[i] = 0.0f;
  }
  if (tid == 0) S.loss = 0.0f;
  const float invA8 = 1.0f / (8.0f * (float)max(A, 1));
  const float invA4 = 1.0f / (4.0f * (float)max(A, 1));
  const float* W1 = S.w + OFF_W1;
  const float* b1 = S.w + OFF_B1;
  const float* W2 = S.w + OFF_W2;
  const float* b2 = S.w + OFF_B2;
  const float* W3 = S.w + OFF_W3;
  const float* b3 = S.w + OFF_B3;
  const int64_t ntiles = (n + TR_TILE - 1) / TR_TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * TR_TILE;
    const int cnt = (int)min((int64_t)TR_TILE, n - base);
    __syncthreads();
    // inputs and labels
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
    // h1 = relu(W1 x + b1)
    for (int i = tid; i < TR_TILE * MLP_H; i += TR_THREADS) {
      const int r = i / MLP_H, u = i % MLP_H;
      float a = b1[u];
#pragma unroll 8
      for (int k = 0; k < MLP_IN; ++k) a = fmaf(W1[u * MLP_IN + k], S.x[r][k], a);
      S.h1[r][u] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    // h2 = relu(W2 h1 + b2)
    for (int i = tid; i < TR_TILE * MLP_H; i += TR_THREADS) {
      const int r = i / MLP_H, u = i % MLP_H;
      float a = b2[u];
#pragma unroll 8
      for (int k = 0; k < MLP_H; ++k) a = fmaf(W2[u * MLP_H + k], S.h1[r][k], a);
      S.h2[r][u] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    // z = W3 h2 + b3
    for (int i = tid; i < TR_TILE * MLP_OUT; i += TR_THREADS) {
      const int r = i / MLP_OUT, u = i % MLP_OUT;
      float a = b3[u];
#pragma unroll 8
      for (int k = 0; k < MLP_H; ++k) a = fmaf(W3[u * MLP_H + k], S.h2[r][k], a);
      S.dz[r][u] = a;
    }
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
      if (ok) atomicAdd(&S.loss, l * scale);
    }
    __syncthreads();
    // d2 = (W3^T dz) * [h2 > 0]
    for (int i = tid; i < TR_TILE * MLP_H; i += TR_THREADS) {
      const int r = i / MLP_H, k = i % MLP_H;
      float a = 0.0f;
#pragma unroll
      for (int u = 0; u < MLP_OUT; ++u) a = fmaf(W3[u * MLP_H + k], S.dz[r][u], a);
      S.d2[r][k] = S.h2[r][k] > 0.0f ? a : 0.0f;
    }
    // gW3 += dz^T h2, gb3 += sum dz
    for (int i = tid; i < NP_W3 + NP_B3; i += TR_THREADS) {
      float a = 0.0f;
      if (i < NP_W3) {
        const int u = i / MLP_H, k = i % MLP_H;
        for (int r = 0; r < TR_TILE; ++r) a = fmaf(S.dz[r][u], S.h2[r][k], a);
      } else {
        for (int r = 0; r < TR_TILE; ++r) a += S.dz[r][i - NP_W3];
      }
      S.g[OFF_W3 + i] += a;
    }
    __syncthreads();
    // d1 = (W2^T d2) * [h1 > 0]
    for (int i = tid; i < TR_TILE * MLP_H; i += TR_THREADS) {
      const int r = i / MLP_H, k = i % MLP_H;
      float a = 0.0f;
#pragma unroll 8
      for (int u = 0; u < MLP_H; ++u) a = fmaf(W2[u * MLP_H + k], S.d2[r][u], a);
      S.d1[r][k] = S.h1[r][k] > 0.0f ? a : 0.0f;
    }
    // gW2 += d2^T h1, gb2 += sum d2
    for (int i = tid; i < NP_W2 + NP_B2; i += TR_THREADS) {
      float a = 0.0f;
      if (i < NP_W2) {
        const int u = i / MLP_H, k = i % MLP_H;
        for (int r = 0; r < TR_TILE; ++r) a = fmaf(S.d2[r][u], S.h1[r][k], a);
      } else {
        for (int r = 0; r < TR_TILE; ++r) a += S.d2[r][i - NP_W2];
      }
      S.g[OFF_W2 + i] += a;
    }
    __syncthreads();
    // gW1 += d1^T x, gb1 += sum d1
    for (int i = tid; i < NP_W1 + NP_B1; i += TR_THREADS) {
      float a = 0.0f;
      if (i < NP_W1) {
        const int u = i / MLP_IN, k = i % MLP_IN;
        for (int r = 0; r < TR_TILE; ++r) a = fmaf(S.d1[r][u], S.x[r][k], a);
      } else {
        for (int r = 0; r < TR_TILE; ++r) a += S.d1[r][i - NP_W1];
      }
      S.g[OFF_W1 + i] += a;
    }
  }
  __syncthreads();
  for (int i = tid; i < NPARAM; i += TR_THREADS) atomicAdd(grad + i, S.g[i]);
  if (tid == 0) atomicAdd(loss_out, S.loss);
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

extern "C" ks_status ks_bc_grad(const float* params, const int32_t* records, int64_t n, int32_t A, float* grad,
                                float* loss, float scale, void* stream) {
  if (!params || !grad || !loss || n < 0 || (n > 0 && !records) || A < 1) return KS_ERR_INVALID_ARG;
  if (n == 0) return KS_OK;
  const size_t smem = sizeof(ks::TrainSmem);
  if (cudaFuncSetAttribute(ks::bc_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return KS_ERR_CUDA;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (n + ks::TR_TILE - 1) / ks::TR_TILE;
  const int grid = (int)(ntiles < (int64_t)sms ? ntiles : (int64_t)sms);
  ks::bc_grad_kernel<<<grid, ks::TR_THREADS, smem, (cudaStream_t)stream>>>(params, records, n, A, grad, loss, scale);
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
