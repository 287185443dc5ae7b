// ks_plain.cuh -- persistent kernel for ensembles of equal-sized markets: one
// CTA is one market group, markets are dealt to CTAs round-robin.
#pragma once

#include "ks_market.cuh"

namespace ks {

// Register-cap classes of the launch bounds: 0 = compiler's choice, 1 = about
// 85 registers per thread.
template <int NT, int OCC>
struct MinBlocks {
  static constexpr int value = OCC == 0 ? 1 : (65536 / (NT * 85) > 0 ? 65536 / (NT * 85) : 1);
};

template <int NT, int AK, bool AGGR, int OCC>
__global__ void __launch_bounds__(NT, MinBlocks<NT, OCC>::value) plain_kernel(DevParams P, uint32_t n_steps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem sm = carve<NT, AK>(smem_raw, P.Lmax);
  const uint32_t s0 = (uint32_t)(*P.step);
  for (uint32_t m = blockIdx.x; m < P.M; m += gridDim.x)
    run_market<NT, AK, AGGR>(P, m, s0, n_steps, sm, (int)threadIdx.x, 0, P.Lmax);
}

template <int NT, int AK, bool AGGR, int OCC>
cudaError_t launch_plain(const DevParams& p, uint32_t n_steps, int grid, size_t smem, cudaStream_t st) {
  plain_kernel<NT, AK, AGGR, OCC><<<grid, NT, smem, st>>>(p, n_steps);
  return cudaGetLastError();
}

}  // namespace ks
