"""GPU parity of the continuous double auction (ks_cda_*) against the oracle:
order words, accounts, the time-priority successor of every resting order,
market scalars and the per-step trace, bit-exact, on every market."""
import numpy as np
import pytest

import oracle as o
from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _compare(gs, ens, m, mk, tp=None, tv=None, trace_from=0):
    sl = ens.market_slice(m)
    od = ks.unpack_orders(gs["order"][sl])
    assert np.array_equal(od["qty"], mk.qty), f"market {m}: order quantities"
    live = mk.qty > 0
    assert np.array_equal(od["side"][live], mk.side[live]), f"market {m}: sides"
    assert np.array_equal(od["tick"][live], mk.tick[live]), f"market {m}: ticks"
    assert np.array_equal(od["atype"], mk.atype), f"market {m}: classes"
    assert np.array_equal(gs["inventory"][sl], mk.inv), f"market {m}: inventory"
    assert np.array_equal(gs["cash"][sl], mk.cash), f"market {m}: cash"
    assert np.array_equal(gs["next"][sl], o.cda_next(mk)), f"market {m}: time priority"
    sc = mk.scalars()
    assert int(gs["last_tick"][m]) == sc["last"], m
    assert list(gs["history"][m]) == sc["hist"], m
    assert int(gs["fundamental"][m]) == sc["fund"], m
    assert int(gs["fills"][m]) == sc["trades"], m
    assert int(gs["last_volume"][m]) == sc["last_v"], m
    assert int(gs["traded_value"][m]) == sc["sum_p"], m
    assert int(gs["sum_volume"][m]) == sc["sum_v"], m
    assert int(gs["trace_hash"][m]) == sc["hash"], m
    if tp is not None and m < gs["trace"].shape[0]:
        n = len(tp)
        gt = gs["trace"][m, trace_from:trace_from + n]
        assert np.array_equal(gt[:, 0], tp), f"market {m}: last fill ticks at {np.nonzero(gt[:, 0] != tp)[0][:8]}"
        assert np.array_equal(gt[:, 1], tv), f"market {m}: volumes"


def _run(w, steps, splits=None, trace=True):
    ens = ks.CdaEnsemble(w, trace_markets=w["M"] if trace else 0, trace_steps=steps if trace else 0)
    for n in splits or [steps]:
        ens.step(n)
    assert ens.sync(timeout_ms=300_000) == ks.KS_OK
    return ens, ens.read_state()


@pytest.mark.parametrize("L,A", [(256, 300), (1024, 1024), (64, 33)])
def test_every_market_and_step_matches_the_oracle(L, A):
    w = wl.workload("cda_8192", M=10, L=L, A=A)
    steps = 120
    ens, gs = _run(w, steps)
    assert int(gs["step"][0]) == steps
    total = 0
    for m in range(w["M"]):
        mk = o.cda_init(w["params"], m, L, A)
        tp, tv, _ = o.cda_run(w["params"], mk, 0, steps)
        _compare(gs, ens, m, mk, tp, tv)
        total += int(tv.sum())
    assert total > 0


@pytest.mark.parametrize("L,A", [(2, 1), (2, 40), (1000, 31), (4096, 2000), (128, 0), (300, 8192), (4096, 8192)])
def test_edge_shapes(L, A):
    w = wl.workload("cda_8192", M=3, L=L, A=A)
    steps = 60
    ens, gs = _run(w, steps)
    for m in range(w["M"]):
        mk = o.cda_init(w["params"], m, L, A)
        tp, tv, _ = o.cda_run(w["params"], mk, 0, steps)
        _compare(gs, ens, m, mk, tp, tv)


@pytest.mark.parametrize("thr", [0, 0x40000000, 0xC0000000, 0xFFFFFFFF])
def test_cancellation_rates(thr):
    """From no cancellations to every working order cancelled each step: orders
    leave their FIFOs from the head, the middle and the tail."""
    w = wl.workload("cda_8192", M=6, L=128, A=500, cancel_thresh_q32=thr)
    steps = 80
    ens, gs = _run(w, steps)
    for m in range(w["M"]):
        mk = o.cda_init(w["params"], m, 128, 500)
        tp, tv, _ = o.cda_run(w["params"], mk, 0, steps)
        _compare(gs, ens, m, mk, tp, tv)


def test_many_markets_per_cta():
    """Enough markets that each CTA holds several books (one warp each)."""
    w = wl.workload("cda_8192", M=1000, L=64, A=100)
    steps = 40
    ens, gs = _run(w, steps, trace=False)
    for m in range(w["M"]):
        mk = o.cda_init(w["params"], m, 64, 100)
        o.cda_run(w["params"], mk, 0, steps)
        _compare(gs, ens, m, mk)


def test_split_calls_keep_time_priority():
    """The FIFOs persist across calls only through the next indices."""
    w = wl.workload("cda_8192", M=8, L=512, A=700)
    _, a = _run(w, 90)
    _, b = _run(w, 90, splits=[1, 29, 47, 13])
    for f in a:
        assert np.array_equal(a[f], b[f]), f


def test_shard_equals_global_markets():
    k = 5
    ws = dict(wl.workload("cda_8192", M=3, L=256, A=400), market_base=k)
    ens, gs = _run(ws, 50)
    for i in range(3):
        mk = o.cda_init(ws["params"], k + i, 256, 400)
        tp, tv, _ = o.cda_run(ws["params"], mk, 0, 50)
        _compare(gs, ens, i, mk, tp, tv)


def test_full_size_sampled_markets():
    w = wl.workload("cda_8192")
    S = int(w["S"])
    ens, gs = _run(w, S, trace=False)
    for m in (0, 1, 4097, 8191):
        mk = o.cda_init(w["params"], m, int(w["L"]), int(w["A"]))
        o.cda_run(w["params"], mk, 0, S)
        _compare(gs, ens, m, mk)


def test_invalid_configs_are_refused():
    for over, st in ((dict(A=8193), ks.KS_ERR_UNSUPPORTED), (dict(L=1), ks.KS_ERR_UNSUPPORTED),
                     (dict(mix_pct=(50, 20, 20)), ks.KS_ERR_INVALID_ARG)):
        w = wl.workload("cda_8192", M=2, **over)
        with pytest.raises(ks.KsError) as ei:
            ks.CdaEnsemble(w)
        assert ei.value.status == st
