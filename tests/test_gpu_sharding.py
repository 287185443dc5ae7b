"""Sharding correctness on one GPU: markets are independent (Sec. III-A) and
every draw is keyed by the global market index, so an ensemble created with
market_base = k must hold exactly global markets k .. k+M-1: equal to the
oracle's markets of those indices and to the matching markets of an
unsharded run, bit for bit.  This is the only correctness claim a
collective-free split of the markets over GPUs needs.  Covered for the
plain kernel, the batched kernel and the paper-agent kernel."""
import numpy as np
import pytest

import oracle as o
from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

from helpers import compare_market

pytestmark = pytest.mark.gpu

AGENT_FIELDS = ("order", "inventory", "cash")
MARKET_FIELDS = ("last_tick", "history", "fundamental", "trades", "last_volume", "sum_price", "sum_volume",
                 "trace_hash")


def _run(w, steps, L=None, A=None, trace=True):
    ens = ks.Ensemble(w, trace_markets=w["M"] if trace else 0, trace_steps=steps if trace else 0, L=L, A=A)
    ens.step(steps)
    assert ens.sync(timeout_ms=600_000) == ks.KS_OK
    return ens, ens.read_state()


def _same_markets(full, gf, part, gp, k):
    for i in range(part.M):
        a, b = full.market_slice(k + i), part.market_slice(i)
        for f in AGENT_FIELDS:
            assert np.array_equal(gf[f][a], gp[f][b]), (k, i, f)
        for f in MARKET_FIELDS:
            assert np.array_equal(gf[f][k + i], gp[f][i]), (k, i, f)
        assert np.array_equal(gf["trace"][k + i], gp["trace"][i]), (k, i)


@pytest.mark.parametrize("k", [1, 5])
def test_plain_shard_equals_global_markets(k):
    steps, M = 60, 8
    w = wl.workload("plain_mix_8192", M=M, L=256, A=640)
    full, gf = _run(w, steps)
    ws = dict(wl.workload("plain_mix_8192", M=3, L=256, A=640), market_base=k)
    part, gp = _run(ws, steps)
    _same_markets(full, gf, part, gp, k)
    for i in range(3):
        mk = o.init_market(w["params"], k + i, 256, 640)
        tp, tv = o.run_market(w["params"], mk, 0, steps)
        compare_market(gp, part, i, mk, tp, tv)


def test_batched_shard_equals_global_markets():
    """Uneven markets: the shard takes the (L, A) of global markets k.. and must
    reproduce them through the batched kernel."""
    steps, M, k, n = 40, 24, 9, 6
    L, A = wl.batched_sizes(M, seed=13)
    A = np.minimum(A, 4096).astype(np.int32)
    w = wl.workload("batched_20000", M=M)
    full, gf = _run(w, steps, L=L, A=A)
    ws = dict(wl.workload("batched_20000", M=n), market_base=k)
    part, gp = _run(ws, steps, L=L[k:k + n], A=A[k:k + n])
    assert part.batch_info()["batched"] == 1
    _same_markets(full, gf, part, gp, k)
    for i in range(n):
        mk = o.init_market(w["params"], k + i, int(L[k + i]), int(A[k + i]))
        tp, tv = o.run_market(w["params"], mk, 0, steps)
        compare_market(gp, part, i, mk, tp, tv)


def test_paper_agent_shard_equals_global_markets():
    steps, M, k, n = 80, 12, 7, 4
    w = wl.workload("paper_8192_256", M=M, L=128, A=256)
    ws = dict(wl.workload("paper_8192_256", M=n, L=128, A=256), market_base=k)
    gf, gp = [], []
    for wk, out in ((w, gf), (ws, gp)):
        ens = ks.PaperEnsemble(wk, trace_markets=wk["M"], trace_steps=steps)
        ens.step(steps)
        assert ens.sync(timeout_ms=300_000) == ks.KS_OK
        out.append(ens.read_state())
        ens.close()
    gf, gp = gf[0], gp[0]
    for i in range(n):
        for f in ("bid", "ask", "last_tick", "mid2", "trades", "last_volume", "sum_price", "sum_volume",
                  "trace_hash", "trace"):
            assert np.array_equal(gf[f][k + i], gp[f][i]), (i, f)
        bk = o.paper_init(k + i, 128, 256)
        tp, tv = o.paper_run(w["params"], bk, 0, steps)
        assert np.array_equal(gp["trace"][i, :, 0], tp) and np.array_equal(gp["trace"][i, :, 1], tv), i
        assert int(gp["trace_hash"][i]) == bk.scalars()["hash"], i
