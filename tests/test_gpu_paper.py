"""GPU parity of the paper-agent kernel (the paper's own NOISE / MOMENTUM /
MAKER agents on a tick-aggregated book) against the oracle: the clearing
trace of every step, the resting book and the market scalars, bit-exact."""
import numpy as np
import pytest

import oracle as o
from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _check_market(params, gs, m, L, A, steps, s0=0, trace=True):
    bk = o.paper_init(m, L, A)
    tp, tv = o.paper_run(params, bk, s0, steps)
    if trace:
        assert np.array_equal(gs["trace"][m, :steps, 0], tp), m
        assert np.array_equal(gs["trace"][m, :steps, 1], tv), m
    assert np.array_equal(gs["bid"][m], bk.bid), m
    assert np.array_equal(gs["ask"][m], bk.ask), m
    sc = bk.scalars()
    assert int(gs["last_tick"][m]) == sc["last"] and int(gs["mid2"][m]) == sc["mid2"], m
    assert int(gs["trades"][m]) == sc["trades"] and int(gs["last_volume"][m]) == sc["last_v"], m
    assert int(gs["sum_price"][m]) == sc["sum_p"] and int(gs["sum_volume"][m]) == sc["sum_v"], m
    assert int(gs["trace_hash"][m]) == sc["hash"], m
    if "window_base" in gs:
        assert int(gs["window_base"][m]) == sc["base"], m


def _run(w, steps, splits=None, launch=None, trace=True):
    ens = ks.PaperEnsemble(w, trace_markets=w["M"] if trace else 0, trace_steps=steps if trace else 0)
    if launch:
        ens.set_launch(*launch)
    for n in splits or [steps]:
        ens.step(n)
    assert ens.sync(timeout_ms=300_000) == ks.KS_OK
    gs = ens.read_state()
    ens.close()
    return gs


@pytest.mark.parametrize("L,A", [(128, 256), (100, 300), (64, 1024)])
def test_every_market_and_step_matches_the_oracle(L, A):
    w = wl.workload("paper_8192_256", M=20, L=L, A=A)
    steps = 150
    gs = _run(w, steps)
    assert int(gs["step"][0]) == steps
    for m in range(w["M"]):
        _check_market(w["params"], gs, m, L, A, steps)


def test_launch_shapes_and_split_calls_agree():
    w = wl.workload("paper_8192_256", M=40, L=128, A=256)
    ref = _run(w, 90, trace=False)
    for launch, splits in (((128, 2, 1), [90]), ((256, 1, 1), [90]), ((128, 4, 1), [30, 60]),
                           ((256, 2, 1), [1, 88, 1]), ((512, 16, 1), [90]), ((128, 16, 1), [45, 45]),
                           ((128, 2, 8), [90]), ((128, 8, 6), [60, 30]), ((128, 4, 6), [90]), ((32, 8, 1), [90]),
                           ((32, 8, 6), [40, 50]), ((32, 32, 1), [90]), ((64, 4, 1), [90]), ((64, 8, 1), [30, 60])):
        got = _run(w, 90, splits=splits, launch=launch, trace=False)
        for f in ref:
            assert np.array_equal(ref[f], got[f]), (launch, f)


def test_warp_per_market_shapes_agree():
    w = wl.workload("paper_8192_256", M=37, L=128, A=100)
    ref = _run(w, 80, launch=(128, 1, 1))
    for m in range(w["M"]):
        _check_market(w["params"], ref, m, 128, 100, 80)
    for launch in ((32, 4, 1), (256, 1, 1), (128, 1, 8), (32, 8, 6), (32, 16, 1), (32, 32, 1)):
        got = _run(w, 80, launch=launch, splits=[25, 55])
        for f in ref:
            assert np.array_equal(ref[f], got[f]), (launch, f)
    w = wl.workload("paper_8192_256", M=9, L=128, A=64)
    ref = _run(w, 60, launch=(32, 2, 8))
    got = _run(w, 60, launch=(128, 1, 1))
    for f in ref:
        assert np.array_equal(ref[f], got[f]), f


@pytest.mark.parametrize("over", [dict(tie_rule=1), dict(mom_pct=70, maker_pct=15), dict(mom_pct=0, maker_pct=100),
                                  dict(noise_halfwidth=0, p_mkt_q32=0), dict(noise_halfwidth=40, qmax=255)])
def test_rule_variants_match_the_oracle(over):
    w = wl.workload("paper_8192_256", M=8, L=96, A=200, **over)
    gs = _run(w, 120)
    for m in range(w["M"]):
        _check_market(w["params"], gs, m, 96, 200, 120)


def test_edge_shapes():
    for L, A in ((2, 5), (128, 0), (4096, 64), (7, 3)):
        w = wl.workload("paper_8192_256", M=3, L=L, A=A, noise_halfwidth=min(4, L), maker_half_spread=1)
        gs = _run(w, 40)
        for m in range(3):
            _check_market(w["params"], gs, m, L, A, 40)


def test_full_size_peak_workload_sampled_markets():
    """The paper's peak shape (8192 markets x 1024 agents, L=128, S=500):
    the whole ensemble in the default launch, sampled markets against the oracle."""
    w = wl.workload("paper_8192_1024")
    gs = _run(w, w["S"], trace=False)
    for m in (0, 1, 777, 4096, 8190, 8191):
        _check_market(w["params"], gs, m, 128, 1024, w["S"], trace=False)
    # every market traded and stayed on the grid
    assert gs["trades"].min() > 0 and 0 <= gs["last_tick"].min() and gs["last_tick"].max() < 128


def test_composition_sweep_runs_and_momentum_raises_volatility():
    from paper_2606_21784_gb300 import dynamics
    r = dynamics.sweep(alphas=[0.0, 0.15, 0.5], M=16, S=400)
    f = r["facts"]
    # on a sliding window momentum markets run away: the price level spreads
    assert f[0.5]["price_std"] > 5 * f[0.0]["price_std"] > 0
    assert all(x["volume_per_step"] > 0 and x["volatility"] > 0 for x in f.values())
    # the sweep's markets are the oracle's: one configuration's trace, bit-exact
    w = wl.workload("paper_8192_256", M=16, L=128, A=256, mom_pct=50, maker_pct=15, window=1)
    gs = _run(w, 400)
    _check_market(w["params"], gs, 5, 128, 256, 400)
    # and on a fixed grid
    r = dynamics.sweep(alphas=[0.0, 0.5], M=16, S=400, window=False)
    assert r["facts"][0.5]["volatility"] > r["facts"][0.0]["volatility"] > 0


def _run_engines(w, plan, trace=True):
    """plan: list of (engine, n) with engine 'p' (persistent) or 'n' (naive)."""
    steps = sum(n for _, n in plan)
    ens = ks.PaperEnsemble(w, trace_markets=w["M"] if trace else 0, trace_steps=steps if trace else 0)
    for eng, n in plan:
        (ens.step if eng == "p" else ens.step_naive)(n)
    assert ens.sync(timeout_ms=300_000) == ks.KS_OK
    gs = ens.read_state()
    ens.close()
    return gs


@pytest.mark.parametrize("L,A,over", [(128, 256, {}), (100, 300, {}), (64, 1024, {}), (96, 200, dict(tie_rule=1)),
                                      (7, 3, dict(noise_halfwidth=4, maker_half_spread=1)), (128, 0, {})])
def test_naive_engine_matches_the_oracle(L, A, over):
    """The naive engine (one thread per market, book in global memory, serial
    clearing) against the oracle: every market and step, bit-exact."""
    w = wl.workload("paper_8192_256", M=21, L=L, A=A, **over)
    steps = 120
    gs = _run_engines(w, [("n", steps)])
    assert int(gs["step"][0]) == steps
    for m in range(w["M"]):
        _check_market(w["params"], gs, m, L, A, steps)


def test_engines_mix_on_one_ensemble():
    w = wl.workload("paper_8192_256", M=300, L=128, A=256)
    ref = _run_engines(w, [("p", 90)])
    for plan in ([("n", 90)], [("p", 40), ("n", 30), ("p", 20)], [("n", 1), ("p", 88), ("n", 1)]):
        got = _run_engines(w, plan)
        for f in ref:
            assert np.array_equal(ref[f], got[f]), (plan, f)


def test_naive_engine_full_fixed_workload_equals_persistent():
    """The paper's fixed workload (8192 markets x 256 agents, L=128, S=500):
    the two engines leave identical state in every market."""
    w = wl.workload("paper_8192_256")
    a = _run_engines(w, [("p", w["S"])], trace=False)
    b = _run_engines(w, [("n", w["S"])], trace=False)
    for f in a:
        assert np.array_equal(a[f], b[f]), f
    _check_market(w["params"], b, 4321, 128, 256, w["S"], trace=False)


@pytest.mark.parametrize("L,A,mom,launch", [(64, 256, 30, None), (64, 200, 70, (128, 2, 1)), (128, 1024, 70, None),
                                            (64, 5, 30, (32, 1, 1)), (40, 300, 50, (256, 2, 1))])
def test_sliding_window_matches_the_oracle(L, A, mom, launch):
    """Sliding window (runaway momentum markets, marketable orders at the
    window's edges): every market and step of both engines against the oracle."""
    w = wl.workload("paper_8192_256", M=13, L=L, A=A, mom_pct=mom, window=1)
    steps = 300
    gs = _run(w, steps, splits=[100, 200], launch=launch)
    assert np.abs(gs["window_base"]).max() > L  # the windows travelled
    for m in range(w["M"]):
        _check_market(w["params"], gs, m, L, A, steps)
    for plan in ([("n", steps)], [("p", 120), ("n", 60), ("p", 120)]):
        got = _run_engines(w, plan)
        for f in gs:
            assert np.array_equal(gs[f], got[f]), (plan, f)


@pytest.mark.parametrize("L,A,launch,over", [(128, 16, (16, 1, 1), {}), (128, 13, (16, 1, 1), dict(tie_rule=1)),
                                             (128, 64, (16, 4, 1), {}), (128, 40, (16, 4, 8), dict(mom_pct=50, window=1)),
                                             (128, 32, (16, 2, 8), {}), (128, 1, (16, 2, 1), {}),
                                             (100, 20, (16, 2, 1), {}), (40, 64, (16, 4, 1), dict(window=1))])
def test_half_warp_groups_match_the_oracle(L, A, launch, over):
    """Two markets per warp (16-lane groups, each with its own segment of
    shuffles, reductions and barriers): every market and step of an odd
    number of markets, so one warp's second segment runs out of markets
    first, against the oracle and the one-warp shape."""
    w = wl.workload("paper_8192_256", M=23, L=L, A=A, **over)
    steps = 120
    gs = _run(w, steps, splits=[50, 70], launch=launch)
    for m in range(w["M"]):
        _check_market(w["params"], gs, m, L, A, steps)
    ref = _run(w, steps, launch=(32, 2, 1) if A <= 64 else None)
    for f in ref:
        assert np.array_equal(ref[f], gs[f]), f


def test_default_launch_for_mid_sized_ensembles():
    """513 to 2048 markets of 33 to 512 agents default to two warps per market;
    sampled markets match the oracle every step."""
    w = wl.workload("paper_8192_256", M=700, L=128, A=150)
    ens = ks.PaperEnsemble(w, trace_markets=w["M"], trace_steps=60)
    assert ens.get_launch()["threads"] == 64
    ens.step(60)
    assert ens.sync(timeout_ms=300_000) == ks.KS_OK
    gs = ens.read_state()
    ens.close()
    for m in (0, 1, 349, 698, 699):
        _check_market(w["params"], gs, m, 128, 150, 60)
