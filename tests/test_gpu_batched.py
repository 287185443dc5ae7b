"""Batched uneven ensembles: GPU <-> oracle parity and plan invariance."""
import numpy as np
import pytest

from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

from helpers import compare_market, oracle_markets

pytestmark = pytest.mark.gpu


def _uneven(M, seed=3):
    L, A = wl.batched_sizes(M, seed)
    return L, A


def _run(w, L, A, steps, plan=None, plain=None, trace=0, chunks=None):
    import torch
    ens = ks.Ensemble(w, trace_markets=trace, trace_steps=steps if trace else 0, L=L, A=A)
    if plan is not None:
        ens.set_batch_plan(*plan)
    if plain is not None:
        ens.set_launch(**plain)
    for c in chunks or [steps]:
        ens.step(c)
    assert ens.sync(timeout_ms=600_000) == ks.KS_OK
    torch.cuda.synchronize()
    return ens, ens.read_state()


def test_batched_every_market_vs_oracle():
    M, steps = 48, 60
    L, A = _uneven(M)
    w = wl.workload("batched_20000", M=M)
    ens, gs = _run(w, L, A, steps, trace=M)
    info = ens.batch_info()
    assert info["batched"] == 1 and info["n_items"] >= 1
    ref = oracle_markets(w["params"], range(M), L, A, 0, steps)
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp, tv)


def test_batched_plans_and_plain_agree():
    """Different CTA sizes, group shapes and the plain kernel give identical state."""
    M, steps = 64, 40
    L, A = _uneven(M, seed=11)
    w = wl.workload("batched_20000", M=M)
    _, ref = _run(w, L, A, steps)
    Lm, Am = int(L.max()), int(A.max())
    plans = [
        (512, [(4096, 16384, 512, 32)]),
        (1024, [(4096, 16384, 1024, 16)]),
        (1024, [(512, 256, 32, 8), (512, 1024, 128, 8), (4096, 2048, 256, 8), (4096, 16384, 1024, 16)]),
        (512, [(2048, 256, 64, 4), (2048, 2048, 256, 8), (4096, 16384, 512, 32)]),
    ]
    for plan in plans:
        _, got = _run(w, L, A, steps, plan=plan)
        for f in ref:
            assert np.array_equal(ref[f], got[f]), (plan, f)
    _, got = _run(w, L, A, steps, plain=dict(threads=1024, agents_per_thread=16))
    for f in ref:
        assert np.array_equal(ref[f], got[f]), ("plain", f)


def test_batched_small_markets_many_per_cta():
    """Small markets packed 32 per CTA (one warp each) and 8 per CTA (named barriers)."""
    M, steps = 300, 50
    rng = np.random.default_rng(4)
    L = rng.choice([128, 256], M).astype(np.int32)
    A = rng.integers(1, 250, M).astype(np.int32)
    w = wl.workload("batched_20000", M=M)
    for plan in [(1024, [(256, 256, 32, 8)]), (1024, [(256, 256, 128, 2)]), (512, [(256, 256, 64, 4)])]:
        ens, gs = _run(w, L, A, steps, plan=plan, trace=8)
        ref = oracle_markets(w["params"], range(0, M, 7), L, A, 0, steps)
        for m, (mk, tp, tv) in ref.items():
            compare_market(gs, ens, m, mk, tp if m < 8 else None, tv if m < 8 else None)


def test_batched_graph_capture_and_split():
    import torch
    M = 40
    L, A = _uneven(M, seed=5)
    w = wl.workload("batched_20000", M=M)
    _, ref = _run(w, L, A, 60)
    ens = ks.Ensemble(w, L=L, A=A)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ens.step(20, stream=torch.cuda.current_stream())
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    got = ens.read_state()
    for f in ref:
        if f != "trace":
            assert np.array_equal(ref[f], got[f]), f
    _, split = _run(w, L, A, 60, chunks=[7, 33, 20])
    for f in ref:
        assert np.array_equal(ref[f], split[f]), f


def test_full_size_batched_sampled_markets():
    """20000 uneven markets x 2000 steps in one launch; one market per (L, A) class vs the oracle."""
    from paper_2606_21784_gb300 import autotune
    w = wl.workload("batched_20000")
    L, A = wl.sizes(w)
    ens = ks.Ensemble(w, L=L, A=A)
    ens.step(w["S"])
    assert ens.sync(timeout_ms=900_000) == ks.KS_OK
    gs = ens.read_state()
    classes = autotune.buckets_of(L, A)
    sample = sorted(int(v[len(v) // 2]) for v in classes.values())
    ref = oracle_markets(w["params"], sample, L, A, 0, w["S"])
    for m, (mk, _, _) in ref.items():
        compare_market(gs, ens, m, mk)
    assert int(gs["cash"].sum()) == 0
    assert int(gs["inventory"].astype(np.int64).sum()) == 0


def test_autotuner_plan_is_valid_and_invariant():
    from paper_2606_21784_gb300 import autotune
    M, steps = 80, 30
    L, A = _uneven(M, seed=9)
    w = wl.workload("batched_20000", M=M)
    plan = autotune.tune_batched(w, L, A, steps=5, use_cache=False, check_default=False)
    assert plan["cta_threads"] in (512, 1024) and plan["buckets"]
    # against the default plan on the whole ensemble: a composed plan, or the default kept
    final = autotune.tune_batched(w, L, A, steps=5, use_cache=False)
    assert final["buckets"] is None or len(final["buckets"]) == len(plan["buckets"])
    _, ref = _run(w, L, A, steps)
    _, got = _run(w, L, A, steps, plan=(plan["cta_threads"], plan["buckets"]))
    for f in ref:
        assert np.array_equal(ref[f], got[f]), f


def test_agents_spread_over_a_large_group_edge_sizes():
    """One 512 x 32 bucket for markets of 0 .. 16384 agents: a market gives each
    thread ceil(A / 512) agents (one for A < 512, with most threads empty;
    odd counts pair an agent with an empty slot), and every market and step
    still matches the oracle."""
    A = np.array([0, 1, 31, 33, 511, 513, 1000, 1537, 9000, 16384], np.int32)
    L = np.array([128, 256, 512, 1024, 2048, 128, 256, 1024, 512, 2048], np.int32)
    M, steps = len(A), 30
    w = wl.workload("batched_20000", M=M)
    ens, gs = _run(w, L, A, steps, plan=(512, [(2048, 16384, 512, 32)]), trace=M)
    ref = oracle_markets(w["params"], range(M), L, A, 0, steps)
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp, tv)
