// ks_internal.h -- structures shared by the host library and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kineticsim.h"

namespace ks {

// Per-market scalar block layouts in the workspace.
constexpr int MI32_STRIDE = 16;  // last, hist[9], fund, trades, last_v, pad x3
constexpr int MI_LAST = 0;
constexpr int MI_HIST = 1;
constexpr int MI_FUND = 10;
constexpr int MI_TRADES = 11;
constexpr int MI_LASTV = 12;
constexpr int MI64_STRIDE = 4;  // sum_p, sum_v, hash, pad
constexpr int MI_SUMP = 0;
constexpr int MI_SUMV = 1;
constexpr int MI_HASH = 2;

// Error word bits.
constexpr uint32_t ERR_SHAPE = 1u;      // market larger than the launch shape
constexpr uint32_t ERR_TICK = 2u;       // tick index outside [0, L)
constexpr uint32_t ERR_RANGE = 4u;      // clearing volume outside the packed range
constexpr uint32_t ERR_MLP_WAIT = 8u;   // bounded tensor-core wait gave up

// Everything a kernel needs, passed by value.
struct DevParams {
  uint32_t M;
  uint32_t market_base;  // global index of market 0 (Philox counter word)
  int32_t L_all, A_all;
  uint32_t key0, key1;
  uint32_t rk[20];       // Philox round keys: rk[2r] = key0 + r * 0x9E3779B9, rk[2r+1] = key1 + r * 0xBB67AE85
  int32_t carry;
  uint32_t cancel_thr;
  uint32_t mix0, mix01;  // class percentile thresholds: ZI < mix0 <= MOM < mix01 <= MR
  int32_t zi_off, zi_qmax, mom_lb, mom_omax, mr_omax, rb_qmax;
  uint32_t mlp_pct;
  int32_t mlp_tile_wgs;  // plain policy kernels: warpgroups of a CTA that evaluate policy tiles
  int32_t tie_rule;
  uint32_t trace_markets, trace_steps;
  int32_t Lmax;  // largest L in the ensemble (shared-memory sizing)

  uint32_t* slot;
  int32_t* inv;
  int64_t* cash;
  int32_t* mi32;  // [M][MI32_STRIDE]
  int64_t* mi64;  // [M][MI64_STRIDE]
  const int64_t* agent_off;  // [M+1] or nullptr (uniform: m*A_all)
  const int32_t* Ls;         // [M] or nullptr
  const int32_t* As;         // [M] or nullptr
  int32_t* trace;            // [trace_markets][trace_steps][2]
  uint32_t* err;
  const uint64_t* step;      // absolute step counter (device)

  // learned agents and captures (used by the kernels compiled with the policy path)
  const unsigned char* mlp;  // policy parameter blob or nullptr
  int32_t* rec;              // rule-decision records [rec_cap][KS_RECORD_WORDS]
  unsigned long long* rec_count;
  uint64_t rec_cap;
  uint32_t rec_agents;       // record agents a < rec_agents of every market
  uint32_t* dec_trace;       // [trace_steps][dec_trace_agents] policy decisions of traced markets
  unsigned long long* pol_count;  // policy decisions evaluated
  uint64_t dec_trace_agents; // agents of markets 0..trace_markets-1
  float* logit_trace;        // [trace_steps][dec_trace_agents][MLP_OUT] policy logits of traced markets
};

// A persistent launch of the plain kernel template.
using PlainLaunchFn = cudaError_t (*)(const DevParams& p, uint32_t n_steps, int grid, size_t smem, cudaStream_t st);
struct PlainVariant {
  int threads;
  int ak;
  int aggregate;  // warp-aggregated book atomics
  int occupancy;  // register-cap class (0 none, 1 128, 2 85 registers per thread)
  PlainLaunchFn launch;
  const void* kernel;  // for attribute and occupancy queries
  int mlp = 0;         // policy path compiled in
  int spread = 0;      // a market's agents spread over the CTA (ceil(A / threads) per thread)
  int carried = 0;     // compiled for carried books only (else the book mode is read at run time)
};

// Registry filled by the instantiation translation units.
const PlainVariant* find_plain(int threads, int ak, int aggregate, int occupancy, bool mlp);
// The spreading rule-agent variant of a shape, or nullptr where none is compiled.
const PlainVariant* find_plain_spread(int threads, int ak, int occupancy);
// The carried-book variant of a full rule-agent shape, or nullptr where none is compiled.
const PlainVariant* find_plain_carried(int threads, int ak, int occupancy);

}  // namespace ks

