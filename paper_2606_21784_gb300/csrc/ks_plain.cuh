// ks_plain.cuh -- persistent kernel for ensembles of equal-sized markets: one
// CTA is one market group, markets are dealt to CTAs round-robin.
#pragma once

#include "ks_market.cuh"

namespace ks {

// Thread 0 of a CTA prefetches into L2 the state of the market it runs next
// (order words, inventory, cash and scalars), so that the next market's state
// loads find it there: the load of market m + grid overlaps market m.
__device__ __forceinline__ void prefetch_next_market(const DevParams& P, uint32_t m) {
  const uint32_t n = m + gridDim.x;
  if (threadIdx.x != 0 || n >= P.M) return;
  const int A = P.As ? P.As[n] : P.A_all;
  const int64_t aoff = P.agent_off ? P.agent_off[n] : (int64_t)n * (int64_t)P.A_all;
  if (A <= 0) return;
  l2_prefetch(P.slot + aoff, (size_t)A * 4);
  l2_prefetch(P.inv + aoff, (size_t)A * 4);
  l2_prefetch(P.cash + aoff, (size_t)A * 8);
  l2_prefetch(P.mi32 + (size_t)n * MI32_STRIDE, MI32_STRIDE * 4);
  l2_prefetch(P.mi64 + (size_t)n * MI64_STRIDE, MI64_STRIDE * 8);
}

// Register-cap classes of the launch bounds: 0 = compiler's choice, 1 = 128
// registers per thread (two 256-thread CTAs per SM), 2 = 85 (three), 3 = 64
// (32 warps per SM: two 512-thread CTAs or one 1024-thread CTA).
// Returns the launch bounds' minimum of resident CTAs.
__host__ __device__ constexpr int plain_cap_regs(int occ) { return occ == 2 ? 85 : (occ == 3 ? 64 : 128); }
__host__ __device__ constexpr int plain_min_ctas(int nt, int occ) {
  return occ == 0 ? 1 : (65536 / (nt * plain_cap_regs(occ)) > 0 ? 65536 / (nt * plain_cap_regs(occ)) : 1);
}

// SPREAD: each market spreads its agents over the CTA (ceil(A / NT) per
// thread) instead of AK per thread, so a market smaller than the shape's
// capacity takes fewer passes; the state is the same bit for bit.
// CM: 2 reads the book mode from the parameters; 1 is compiled for carried
// books only (the host launches it only for an ensemble that carries them).
template <int NT, int AK, bool AGGR, int OCC, bool MLP = false, bool SPREAD = false, int CM = 2>
__global__ void __launch_bounds__(NT, plain_min_ctas(NT, OCC)) plain_kernel(DevParams P, uint32_t n_steps) {
  constexpr int BUDGET = thread_reg_budget(NT, plain_min_ctas(NT, OCC));
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const uint32_t s0 = (uint32_t)(*P.step);
  if constexpr (MLP) {
    // policy path: weights, then the market group; warpgroups 0 .. tile_wgs-1
    // evaluate policy tiles, each with MLP_TMEM_COLS TMEM columns (its
    // accumulator and activations), an mbarrier and a named barrier
    constexpr int NWG = NT / 128;
    const int twg = min(max(P.mlp_tile_wgs, 1), min(NWG, MLP_MAX_TILE_WGS));
    const MlpCta mc = mlp_cta_carve(smem_raw, (uint32_t)twg * MLP_TMEM_COLS);
    mlp_cta_setup(mc, P.mlp);
    unsigned char* graw = smem_raw + mlp_cta_bytes();
    const Smem sm = carve<NT, AK, true, true>(graw, P.Lmax);
    const int wg = (int)threadIdx.x / 128;
    MlpWG mw;
    mw.wg = wg;
    mw.nwg = twg;
    mw.bar = &mc.bars[wg];
    mw.tmem = *mc.tslot + (uint32_t)(min(wg, twg - 1) * MLP_TMEM_COLS);
    mw.bar_id = 1 + wg;
    mw.phase = 0;
    mw.abort = false;
    for (uint32_t m = blockIdx.x; m < P.M; m += gridDim.x) {
      prefetch_next_market(P, m);
      run_market<NT, AK, false, true, false>(P, m, s0, n_steps, sm, (int)threadIdx.x, 0, P.Lmax, &mw, mc.sw);
    }
    mlp_cta_teardown(mc);
  } else {
    constexpr bool REGACC = accounts_in_registers(BUDGET, AK, false);
    const Smem sm = carve<NT, AK, false, !REGACC>(smem_raw, P.Lmax);
    for (uint32_t m = blockIdx.x; m < P.M; m += gridDim.x) {
      prefetch_next_market(P, m);
      run_market<NT, AK, AGGR, false, REGACC, SPREAD, CM>(P, m, s0, n_steps, sm, (int)threadIdx.x, 0, P.Lmax);
    }
  }
}

template <int NT, int AK, bool AGGR, int OCC, bool MLP = false, bool SPREAD = false, int CM = 2>
cudaError_t launch_plain(const DevParams& p, uint32_t n_steps, int grid, size_t smem, cudaStream_t st) {
  plain_kernel<NT, AK, AGGR, OCC, MLP, SPREAD, CM><<<grid, NT, smem, st>>>(p, n_steps);
  return cudaGetLastError();
}

// Dynamic shared memory of a plain launch (occ: register-cap class; policy
// kernels add the weights, their activations live in TMEM).
__host__ __device__ inline size_t plain_launch_smem(int nt, int ak, int occ, int Lmax, bool mlp) {
  size_t o[8];
  const size_t m = group_smem_layout(thread_reg_budget(nt, plain_min_ctas(nt, occ)), nt, ak, Lmax, mlp, o);
  return mlp ? mlp_cta_bytes() + m : m;
}

}  // namespace ks
