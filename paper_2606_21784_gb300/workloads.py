"""Seeded synthetic workloads: ensemble sizes and agent parameters.

This module only describes inputs.  It holds none of the method's arithmetic,
so both the CUDA library and the CPU oracle can be driven from it.

Five workloads, one per benchmark configuration of the method:

``plain_zi_64``     64 markets, L=256, A=256, S=1000, zero-intelligence agents,
                    unfilled orders discarded every step.
``plain_mix_8192``  8192 markets, L=1024, A=4096, S=2000, 60/20/20 mix of
                    zero-intelligence / momentum / mean-reversion agents,
                    carried book with per-order cancellation 0.05.
``batched_20000``   20000 markets, L in {128..2048}, A log-uniform in
                    [64, 16384], S=2000, agents as ``plain_mix_8192``.
``learned_4096``    4096 markets, L=512, A=2048, S=2000, all agents MLP-driven.
``mixed_32768``     32768 markets, L in {256..2048}, A log-uniform in
                    [128, 8192], S=10000, 25% MLP agents.

The continuous double auction (``CdaEnsemble``; the paper names it as a market
the same pattern extends to) with the configuration's agents:

``cda_8192``        8192 markets, L=1024, A=1024, S=500, agents as ``plain_mix_8192``.

The paper's own agent model (tick-aggregated book, NOISE / MOMENTUM / MAKER
agents around the mid price, SplitMix64 draws; ``PaperEnsemble``) on the
shapes of the paper's throughput tables (L=128, S=500):

``paper_8192_1024`` 8192 markets, A=1024 (the paper's peak configuration).
``paper_8192_256``  8192 markets, A=256 (the paper's fixed workload).

The paper does not publish Delta_noise, P_mkt, q_max or Delta_maker; the
values below are chosen here (the standard mix alpha_mom = 0.15,
alpha_maker = 0.15 is the paper's).

The uneven ensembles draw (L, A) per market from numpy's PCG64 with a fixed
instance seed; the simulation seed is separate.
"""
from __future__ import annotations

import copy

import numpy as np

# round(0.05 * 2^32): a working order is cancelled when its draw word is below this
CANCEL_005_Q32 = 214748365

_ZI_DISCARD = dict(
    seed=1, carry_book=0, cancel_thresh_q32=0, mix_pct=(100, 0, 0),
    zi_offset=16, zi_qmax=10, mom_lookback=8, mom_offset_max=8, mr_offset_max=8, rb_qmax=10,
    mlp_pct=0, tie_rule=0,
)
_MIX_CARRY = dict(
    seed=1, carry_book=1, cancel_thresh_q32=CANCEL_005_Q32, mix_pct=(60, 20, 20),
    zi_offset=32, zi_qmax=100, mom_lookback=8, mom_offset_max=8, mr_offset_max=8, rb_qmax=100,
    mlp_pct=0, tie_rule=0,
)

_PAPER_AGENTS = dict(
    seed=1, noise_halfwidth=4, p_mkt_q32=CANCEL_005_Q32, qmax=10, maker_half_spread=1, mom_pct=15, maker_pct=15,
    tie_rule=0, window=0,
)

WORKLOADS = {
    "plain_zi_64": dict(M=64, L=256, A=256, S=1000, params=_ZI_DISCARD),
    "plain_mix_8192": dict(M=8192, L=1024, A=4096, S=2000, params=_MIX_CARRY),
    "batched_20000": dict(M=20000, L=None, A=None, S=2000, params=_MIX_CARRY,
                          instance=dict(kind="batched", seed=3)),
    "learned_4096": dict(M=4096, L=512, A=2048, S=2000, params=dict(_MIX_CARRY, mlp_pct=100)),
    "mixed_32768": dict(M=32768, L=None, A=None, S=10000, params=dict(_MIX_CARRY, mlp_pct=25),
                        instance=dict(kind="mixed", seed=5)),
    "cda_8192": dict(M=8192, L=1024, A=1024, S=500, params=_MIX_CARRY, model="cda"),
    "paper_8192_1024": dict(M=8192, L=128, A=1024, S=500, params=_PAPER_AGENTS, model="paper"),
    "paper_8192_256": dict(M=8192, L=128, A=256, S=500, params=_PAPER_AGENTS, model="paper"),
}


def workload(name: str, **overrides) -> dict:
    """A deep copy of a named workload with top-level or ``params`` overrides."""
    w = copy.deepcopy(WORKLOADS[name])
    w["params"] = dict(w["params"])
    for k, v in overrides.items():
        if k in w["params"]:
            w["params"][k] = v
        else:
            w[k] = v
    return w


def batched_sizes(M: int, seed: int = 3):
    """L = 128 * 2^k, k uniform on {0..4}; A = floor(64 * 256^u), u uniform on [0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(0, 5, size=M)
    u = rng.random(M)
    L = (128 * (2 ** k)).astype(np.int32)
    A = np.floor(64.0 * np.power(256.0, u)).astype(np.int32)
    return L, A


def mixed_sizes(M: int, seed: int = 5):
    """L uniform on {256, 512, 1024, 2048}; A = floor(128 * 64^u), u uniform on [0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(0, 4, size=M)
    u = rng.random(M)
    L = (256 * (2 ** k)).astype(np.int32)
    A = np.floor(128.0 * np.power(64.0, u)).astype(np.int32)
    return L, A


def sizes(w: dict):
    """Per-market (L, A) int32 arrays for workload dict ``w``."""
    M = int(w["M"])
    inst = w.get("instance")
    if inst is None:
        return np.full(M, int(w["L"]), np.int32), np.full(M, int(w["A"]), np.int32)
    if inst["kind"] == "batched":
        return batched_sizes(M, inst["seed"])
    if inst["kind"] == "mixed":
        return mixed_sizes(M, inst["seed"])
    raise ValueError(inst["kind"])
