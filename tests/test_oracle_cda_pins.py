"""Pins of the oracle's continuous double auction (readings C1-C6 in the
oracle's header): hand-built books with injected arrivals whose fills are
written out by hand, and invariants of long random runs (conservation,
an uncrossed book, every fill at the resting order's tick and inside the
arriving order's limit, fills of one arrival in price order)."""
import numpy as np
import pytest

import oracle as o

BUY, SELL = 0, 1


def _params(**over):
    from paper_2606_21784_gb300 import workloads as wl
    p = dict(wl.workload("plain_mix_8192")["params"], cancel_thresh_q32=0)
    p.update(over)
    return p


def _book(A, L, resting, last=9):
    """A CDA market whose resting orders are {agent: (side, tick, qty, stamp)}."""
    p = _params()
    mk = o.cda_init(p, 0, L, A)
    mk.qty[:] = 0
    for a, (sd, tk, q, st) in resting.items():
        mk.side[a], mk.tick[a], mk.qty[a], mk.stamp[a] = sd, tk, q, st
    mk.sc.last = last
    return p, mk


def _inject(A, steps, orders):
    """orders: {(step, agent): (side, tick, qty)}; every other decision is no order."""
    d = {k: np.zeros((steps, A), np.int32) for k in ("side", "tick", "qty")}
    for (j, a), (sd, tk, q) in orders.items():
        d["side"][j, a], d["tick"][j, a], d["qty"][j, a] = sd, tk, q
    return d


def test_price_then_time_priority_by_hand():
    """Asks: agents 7 (stamp 2, qty 3) and 3 (stamp 5, qty 4) at tick 10, agent 5
    (qty 6) at 11, agent 9 (qty 5) at 13; bids: agent 1 (qty 2) at 8, agent 2
    (qty 5) at 7.  Agent 0 arrives with a buy of 10 at 11: it takes 3 from agent
    7 and 4 from agent 3 at 10 (time priority), then 3 from agent 5 at 11 (price
    priority before agent 9, which is beyond the limit).  Agent 4 then sells 4 at
    8: 2 from agent 1 at 8, the other 2 rest at 8 (agent 2's bid at 7 does not
    cross)."""
    A, L = 10, 32
    p, mk = _book(A, L, {7: (SELL, 10, 3, 2), 3: (SELL, 10, 4, 5), 5: (SELL, 11, 6, 1), 9: (SELL, 13, 5, 0),
                         1: (BUY, 8, 2, 3), 2: (BUY, 7, 5, 4)})
    inj = _inject(A, 1, {(0, 0): (BUY, 11, 10), (0, 4): (SELL, 8, 4)})
    tp, tv, fills = o.cda_run(p, mk, 0, 1, fills_cap=16, inject=inj)
    assert fills.tolist() == [[0, 0, 7, 10, 3], [0, 0, 3, 10, 4], [0, 0, 5, 11, 3], [0, 4, 1, 8, 2]]
    assert list(mk.inv) == [10, 2, 0, -4, -2, -3, 0, -3, 0, 0]
    assert list(mk.cash) == [-(30 + 40 + 33), -16, 0, 40, 16, 33, 0, 30, 0, 0]
    assert list(mk.qty) == [0, 0, 5, 0, 2, 3, 0, 0, 0, 5]
    assert (mk.side[4], mk.tick[4], mk.stamp[4]) == (SELL, 8, 4)  # arrival stamp s * A + a
    assert mk.stamp[5] == 1 and mk.stamp[0] == -1 and mk.stamp[7] == -1
    assert list(tp) == [8] and list(tv) == [12]  # the step's last fill and its volume
    sc = mk.scalars()
    assert sc["last"] == 8 and sc["trades"] == 4 and sc["sum_p"] == 30 + 40 + 33 + 16 and sc["sum_v"] == 12
    assert sc["hist"][0] == 8 and sc["last_v"] == 12


def test_arrivals_queue_behind_earlier_orders_across_steps():
    """Step 0: agents 2 and 6 bid 5 at tick 20 (agent 2 first, lower index).
    Step 1: agent 8 bids 5 at 20 (behind both); agent 3 sells 7 at 19: 5 from
    agent 2 then 2 from agent 6, all at 20; agent 8 keeps its place behind 6."""
    A, L = 10, 64
    p, mk = _book(A, L, {}, last=20)
    inj = _inject(A, 2, {(0, 2): (BUY, 20, 5), (0, 6): (BUY, 20, 5), (1, 8): (BUY, 20, 5), (1, 3): (SELL, 19, 7)})
    tp, tv, fills = o.cda_run(p, mk, 0, 2, fills_cap=16, inject=inj)
    assert fills.tolist() == [[1, 3, 2, 20, 5], [1, 3, 6, 20, 2]]
    assert list(tp) == [-1, 20] and list(tv) == [0, 7]
    assert mk.qty[6] == 3 and mk.qty[8] == 5 and mk.qty[2] == 0 and mk.qty[3] == 0
    assert mk.stamp[6] == 6 and mk.stamp[8] == 1 * A + 8
    nxt = o.cda_next(mk)
    assert nxt[6] == 8 and nxt[8] == -1
    assert mk.scalars()["last"] == 20 and list(mk.inv[[2, 3, 6]]) == [5, -7, 2]


def test_fill_at_the_resting_price_and_limits():
    """A buy limit above the best ask pays the ask (the resting price), and an
    arrival never trades beyond its own limit: the sell at 14 leaves the bid at 12."""
    A, L = 6, 32
    p, mk = _book(A, L, {1: (SELL, 9, 2, 0), 2: (BUY, 12, 3, 1)}, last=10)
    inj = _inject(A, 1, {(0, 0): (BUY, 15, 2), (0, 3): (SELL, 14, 4)})
    tp, tv, fills = o.cda_run(p, mk, 0, 1, fills_cap=8, inject=inj)
    assert fills.tolist() == [[0, 0, 1, 9, 2]]
    assert list(mk.cash[:2]) == [-18, 18]
    assert (mk.qty[3], mk.tick[3], mk.side[3]) == (4, 14, SELL)
    assert mk.qty[2] == 3


def test_cancellation_frees_the_queue_place():
    """A cancelled order leaves the book before the step's arrivals trade, so an
    arrival trades with the next order in time priority."""
    A, L = 40, 64
    p = _params(cancel_thresh_q32=0x80000000)  # half the working orders cancel
    seed = int(p["seed"])
    key = (seed & 0xFFFFFFFF, seed >> 32)
    cancels = [a for a in range(1, A) if int(o.philox4x32_10((0, a, 0, 0), key)[0]) < 0x80000000]
    keeps = [a for a in range(1, A) if a not in cancels]
    assert cancels and keeps
    c, k = cancels[0], keeps[0]
    mk = o.cda_init(p, 0, L, A)
    mk.qty[:] = 0
    for a, st in ((c, 0), (k, 1)):
        mk.side[a], mk.tick[a], mk.qty[a], mk.stamp[a] = SELL, 30, 4, st
    inj = _inject(A, 1, {(0, 0): (BUY, 30, 4)})
    _, _, fills = o.cda_run(p, mk, 0, 1, fills_cap=8, inject=inj)
    assert fills.tolist() == [[0, 0, k, 30, 4]]
    assert mk.qty[c] == 0 and mk.stamp[c] == -1


@pytest.mark.parametrize("seed", [1, 7])
def test_random_runs_keep_the_invariants(seed):
    """The configuration's agents over 120 steps: volume balance and
    conservation, an uncrossed book after every step, all fills of a resting
    order at its one tick (its old tick if it rested before the step and
    still rests), and the fills of one arrival in price order (a buy from the lowest ask up, a sell from the
    highest bid down)."""
    from paper_2606_21784_gb300 import workloads as wl
    p = dict(wl.workload("plain_mix_8192")["params"], seed=seed)
    A, L = 300, 256
    mk = o.cda_init(p, 3, L, A)
    total_fills = 0
    for s in range(120):
        before = {a: (int(mk.side[a]), int(mk.tick[a]), int(mk.qty[a])) for a in range(A) if mk.qty[a] > 0}
        tp, tv, fills = o.cda_run(p, mk, s, 1, fills_cap=5000)
        assert int(mk.inv.sum()) == 0 and int(mk.cash.sum()) == 0
        assert int(tv[0]) == int(fills[:, 4].sum()) if len(fills) else int(tv[0]) == 0
        bids = mk.tick[(mk.qty > 0) & (mk.side == BUY)]
        asks = mk.tick[(mk.qty > 0) & (mk.side == SELL)]
        if len(bids) and len(asks):
            assert bids.max() < asks.min()
        for inc in np.unique(fills[:, 1]) if len(fills) else []:
            f = fills[fills[:, 1] == inc]
            px = f[:, 3]
            # the arriving order took the book from its best price outwards
            assert np.all(np.diff(px) >= 0) or np.all(np.diff(px) <= 0)
        for r in np.unique(fills[:, 2]) if len(fills) else []:
            ticks = np.unique(fills[fills[:, 2] == r, 3])
            assert len(ticks) == 1  # a resting order trades at its one tick
            # still resting from an earlier step (not cancelled and replaced): its old tick
            if int(r) in before and 0 <= mk.stamp[r] < s * A:
                assert int(ticks[0]) == before[int(r)][1]
        total_fills += len(fills)
        if len(fills):
            assert int(tp[0]) == int(fills[-1, 3])
    assert total_fills > 500
