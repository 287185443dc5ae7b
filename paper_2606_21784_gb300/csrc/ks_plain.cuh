// ks_plain.cuh -- persistent kernel for ensembles of equal-sized markets: one
// CTA is one market group, markets are dealt to CTAs round-robin.
#pragma once

#include "ks_market.cuh"

namespace ks {

// Register-cap classes of the launch bounds: 0 = compiler's choice, 1 = about
// 85 registers per thread (policy kernels: 128, so that two 256-thread CTAs
// share an SM).
template <int NT, int OCC, bool MLP = false>
struct MinBlocks {
  static constexpr int cap = MLP ? 128 : 85;
  static constexpr int value = OCC == 0 ? 1 : (65536 / (NT * cap) > 0 ? 65536 / (NT * cap) : 1);
};

template <int NT, int AK, bool AGGR, int OCC, bool MLP = false>
__global__ void __launch_bounds__(NT, (MinBlocks<NT, OCC, MLP>::value)) plain_kernel(DevParams P, uint32_t n_steps) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const uint32_t s0 = (uint32_t)(*P.step);
  if constexpr (MLP) {
    // policy path: weights, mbarrier and 64 TMEM columns, then the market group
    const MlpCta mc = mlp_cta_carve(smem_raw, MLP_TMEM_COLS);
    mlp_cta_setup(mc, P.mlp);
    unsigned char* graw = smem_raw + mlp_cta_bytes();
    size_t o[8];
    const size_t mbytes = market_smem_layout(NT, AK, P.Lmax, true, o);
    const Smem sm = carve<NT, AK, true>(graw, P.Lmax);
    MlpWG mw;
    mw.act = graw + mbytes;
    mw.bar = &mc.bars[0];
    mw.tmem = *mc.tslot;
    mw.bar_id = 1;
    mw.phase = 0;
    mw.abort = false;
    for (uint32_t m = blockIdx.x; m < P.M; m += gridDim.x)
      run_market<NT, AK, false, true>(P, m, s0, n_steps, sm, (int)threadIdx.x, 0, P.Lmax, &mw, mc.sw);
    mlp_cta_teardown(mc);
  } else {
    const Smem sm = carve<NT, AK>(smem_raw, P.Lmax);
    for (uint32_t m = blockIdx.x; m < P.M; m += gridDim.x)
      run_market<NT, AK, AGGR>(P, m, s0, n_steps, sm, (int)threadIdx.x, 0, P.Lmax);
  }
}

template <int NT, int AK, bool AGGR, int OCC, bool MLP = false>
cudaError_t launch_plain(const DevParams& p, uint32_t n_steps, int grid, size_t smem, cudaStream_t st) {
  plain_kernel<NT, AK, AGGR, OCC, MLP><<<grid, NT, smem, st>>>(p, n_steps);
  return cudaGetLastError();
}

// Dynamic shared memory of a plain launch.
__host__ __device__ inline size_t plain_launch_smem(int nt, int ak, int Lmax, bool mlp) {
  size_t o[8];
  const size_t m = market_smem_layout(nt, ak, Lmax, mlp, o);
  return mlp ? mlp_cta_bytes() + m + MLP_ACT_BYTES : m;
}

}  // namespace ks
