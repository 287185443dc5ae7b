"""Shared test helpers: run the oracle over markets and compare with GPU state."""
import numpy as np

import oracle as o
from paper_2606_21784_gb300 import kineticsim as ks


def oracle_markets(params, markets, L, A, s0, n, init_states=None):
    """Run the oracle for each market index in ``markets`` over [s0, s0+n)."""
    out = {}
    for m in markets:
        mk = o.init_market(params, int(m), int(L[m]), int(A[m])) if init_states is None else init_states[m]
        tp, tv = o.run_market(params, mk, s0, n)
        out[int(m)] = (mk, tp, tv)
    return out


def compare_market(gs, ens, m, mk, tp=None, tv=None, trace_from=0):
    """Assert the GPU state of market m equals the oracle's, field by field."""
    sl = ens.market_slice(m)
    od = ks.unpack_orders(gs["order"][sl])
    assert np.array_equal(od["qty"], mk.qty), f"market {m}: order quantities differ"
    live = mk.qty > 0
    assert np.array_equal(od["side"][live], mk.side[live]), f"market {m}: order sides differ"
    assert np.array_equal(od["tick"][live], mk.tick[live]), f"market {m}: order ticks differ"
    assert np.array_equal(od["atype"], mk.atype), f"market {m}: agent classes differ"
    assert np.array_equal(od["mlp"], mk.mlp), f"market {m}: MLP flags differ"
    assert np.array_equal(gs["inventory"][sl], mk.inv), f"market {m}: inventory differs"
    assert np.array_equal(gs["cash"][sl], mk.cash), f"market {m}: cash differs"
    sc = mk.scalars()
    assert int(gs["last_tick"][m]) == sc["last"], f"market {m}: last tick"
    assert list(gs["history"][m]) == sc["hist"], f"market {m}: history"
    assert int(gs["fundamental"][m]) == sc["fund"], f"market {m}: fundamental"
    assert int(gs["trades"][m]) == sc["trades"], f"market {m}: trades"
    assert int(gs["last_volume"][m]) == sc["last_v"], f"market {m}: last volume"
    assert int(gs["sum_price"][m]) == sc["sum_p"], f"market {m}: sum of p*"
    assert int(gs["sum_volume"][m]) == sc["sum_v"], f"market {m}: sum of V*"
    assert int(gs["trace_hash"][m]) == sc["hash"], f"market {m}: trace hash"
    if tp is not None and "trace" in gs and m < gs["trace"].shape[0]:
        n = len(tp)
        gt = gs["trace"][m, trace_from:trace_from + n]
        assert np.array_equal(gt[:, 0], tp), f"market {m}: clearing ticks differ at steps " \
            f"{np.nonzero(gt[:, 0] != tp)[0][:10]}"
        assert np.array_equal(gt[:, 1], tv), f"market {m}: volumes differ"
