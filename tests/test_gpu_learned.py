"""Learned agents on the GPU vs the oracle.

- Recorded rule decisions (the behaviour-cloning data) equal the oracle's
  records (as multisets: the GPU appends them in no fixed order).
- Markets driven by the tensor-core policy: the orders the GPU emitted are
  replayed through the CPU clearing oracle, which must reproduce the GPU state
  bit for bit; the oracle's own fp64 policy decisions are compared with the
  GPU's and the mismatch rate is reported (FP32 vs FP64 sampling can differ
  near a CDF boundary).
"""
import numpy as np
import pytest

import oracle as o
from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

from helpers import compare_market

pytestmark = pytest.mark.gpu

MISMATCH_MAX = 0.02


def _policy(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, scale, (64, 32))
    b1 = rng.normal(0, 0.2, 64)
    W2 = rng.normal(0, scale, (64, 64))
    b2 = rng.normal(0, 0.2, 64)
    W3 = rng.normal(0, scale, (37, 64))
    b3 = rng.normal(0, 0.2, 37)
    b3[2] = -3.0          # rarely pass
    b3[36] = np.log(30.0)  # quantities around 30
    return W1, b1, W2, b2, W3, b3


def _replay_arrays(dec, A, off):
    """Decision words [steps, traced agents] -> oracle replay arrays for one market."""
    d = dec[:, off:off + A].astype(np.int64) & 0xFFFFFFFF
    none = d == 0xFFFFFFFF
    pas = (d & ks.KS_DECISION_PASS) != 0
    side = np.where(pas, 2, (d >> 8) & 1)
    side = np.where(none, -1, side).astype(np.int32)
    return dict(side=side, tick=((d >> 9) & 0xFFF).astype(np.int32), qty=(d & 0xFF).astype(np.int32))


def test_recorded_rule_decisions_match_oracle():
    import torch
    w = wl.workload("plain_mix_8192", M=4, L=512, A=1024, seed=7)
    steps, rec_agents = 60, 64
    ens = ks.Ensemble(w, trace_markets=4, trace_steps=steps)
    ens.set_capture(record_agents=rec_agents, record_capacity=200000)
    ens.step(steps)
    assert ens.sync(timeout_ms=300_000) == ks.KS_OK
    gpu = ens.records()
    gs = ens.read_state()
    ref = []
    for m in range(4):
        mk = o.init_market(w["params"], m, 512, 1024)
        stats = {}
        tp, tv = o.run_market(w["params"], mk, 0, steps, rec_agents=rec_agents, rec_cap=200000, stats=stats)
        ref.append(stats["records"])
        compare_market(gs, ens, m, mk, tp, tv)
    ref = np.concatenate(ref)
    assert len(gpu) == len(ref) > 1000
    key = lambda r: np.lexsort(r.T[::-1])  # noqa: E731
    assert np.array_equal(gpu[key(gpu)], ref[key(ref)])
    torch.cuda.synchronize()


@pytest.mark.parametrize("mlp_pct,M,L,A,launch", [(100, 6, 512, 2048, None), (25, 5, 1024, 1500, None),
                                                  (100, 6, 512, 2048, (256, 8, 1)), (25, 5, 1024, 1500, (128, 16, 1))])
def test_policy_markets_replay_through_oracle(mlp_pct, M, L, A, launch):
    """launch: (threads, agents per thread, reg_cap); reg_cap 1 is the 128-register policy kernel."""
    import torch
    P = _policy(1)
    blob = ks.pack_mlp_params(*P)
    w = wl.workload("learned_4096", M=M, L=L, A=A, mlp_pct=mlp_pct)
    steps = 40
    ens = ks.Ensemble(w, trace_markets=M, trace_steps=steps, mlp_params=blob)
    ens.set_capture(decisions=True)
    if launch:
        ens.set_launch(launch[0], launch[1], reg_cap=launch[2])
    ens.step(steps)
    assert ens.sync(timeout_ms=300_000) == ks.KS_OK
    gs = ens.read_state()
    dec = ens.capture["decisions"].cpu().numpy()
    w64 = o.mlp_pack(*ks.mlp_params_as_used(*P))
    checked = mism = 0
    for m in range(M):
        mk = o.init_market(w["params"], m, L, A)
        stats = {}
        tp, tv = o.run_market(w["params"], mk, 0, steps, replay=_replay_arrays(dec, A, m * A), mlp_w=w64,
                              stats=stats)
        compare_market(gs, ens, m, mk, tp, tv)
        checked += stats["mlp_checked"]
        mism += stats["mlp_mismatch"]
    assert checked > 1000
    rate = mism / checked
    print(f"policy decisions checked {checked}, mismatch rate {rate:.5f}")
    assert rate <= MISMATCH_MAX
    torch.cuda.synchronize()


def test_policy_batched_uneven_replay():
    import torch
    P = _policy(2)
    blob = ks.pack_mlp_params(*P)
    M, steps = 12, 30
    rng = np.random.default_rng(6)
    L = rng.choice([256, 512, 1024, 2048], M).astype(np.int32)
    A = np.floor(128 * 64.0 ** rng.random(M)).astype(np.int32)
    w = wl.workload("mixed_32768", M=M)
    ens = ks.Ensemble(w, trace_markets=M, trace_steps=steps, L=L, A=A, mlp_params=blob)
    assert ens.batch_info()["batched"] == 1
    ens.set_capture(decisions=True)
    ens.step(steps)
    assert ens.sync(timeout_ms=300_000) == ks.KS_OK
    gs = ens.read_state()
    dec = ens.capture["decisions"].cpu().numpy()
    w64 = o.mlp_pack(*ks.mlp_params_as_used(*P))
    checked = mism = 0
    for m in range(M):
        mk = o.init_market(w["params"], m, int(L[m]), int(A[m]))
        stats = {}
        tp, tv = o.run_market(w["params"], mk, 0, steps,
                              replay=_replay_arrays(dec, int(A[m]), int(ens.offsets[m])), mlp_w=w64, stats=stats)
        compare_market(gs, ens, m, mk, tp, tv)
        checked += stats["mlp_checked"]
        mism += stats["mlp_mismatch"]
    assert checked > 100 and mism / checked <= MISMATCH_MAX
    torch.cuda.synchronize()
