"""Pins of the oracle's paper-agent mode (the paper's own NOISE / MOMENTUM /
MAKER agents on a tick-aggregated book, Sec. III-C, with SplitMix64 draws,
Sec. III-G).

Expected values come from the published SplitMix64 sequence, from the rules
as the paper states them (checked as properties of many draws, not by
re-evaluating the oracle's formulas) and from invariants of a uniform-price
call auction that fix the residual book uniquely.
"""
import os

import numpy as np
import pytest

import oracle as o

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1

BASE = dict(seed=11, noise_halfwidth=4, p_mkt_q32=int(round(0.05 * 2**32)), qmax=10, maker_half_spread=1,
            mom_pct=15, maker_pct=15, tie_rule=0)


def _golden():
    with open(os.path.join(GOLD, "splitmix64_sequence.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    return {int(k): int(v, 16) for k, v in rows}


def _nearest_even_ok(tick, x2, L):
    """tick is x2/2 rounded to the nearest integer with ties to even, clamped to [0, L)."""
    if x2 % 2 == 0:
        r = x2 // 2
    else:  # exactly halfway between (x2 - 1)/2 and (x2 + 1)/2: the even one
        lo = (x2 - 1) // 2
        r = lo if lo % 2 == 0 else lo + 1
    return tick == min(max(r, 0), L - 1)


# --------------------------------------------------------------------------
# draws
# --------------------------------------------------------------------------
def test_draws_follow_the_published_splitmix64_sequence():
    g = _golden()
    # generator state 0: the counter of (gid 0, step 0, channel c) is c
    for c in (1, 2, 3):
        assert o.splitmix64_draw(0, 0, 0, c) == g[c]
    # the seed is the generator state: state k*gamma, counter 1 gives output k + 1
    assert o.splitmix64_draw(GAMMA, 0, 0, 1) == g[2]
    assert o.splitmix64_draw(2 * GAMMA % (1 << 64), 0, 0, 1) == g[3]
    # counter layout gid * 2^35 + 8 step + channel: choose the state so that
    # the draw lands on output 3 of the state-0 sequence
    for gid, s, c in ((1, 0, 0), (5, 7, 1), (123456, 99, 2), (3, 2**20, 0)):
        counter = gid * 2**35 + 8 * s + c
        seed = ((3 - counter) * GAMMA) & M64
        assert o.splitmix64_draw(seed, gid, s, c) == g[3]


def test_class_mix():
    n = 20000
    cls = np.array([o.paper_class(BASE, gid) for gid in range(n)])
    assert abs(np.mean(cls == o.PAPER_MAKER) - 0.15) < 0.015
    assert abs(np.mean(cls == o.PAPER_MOMENTUM) - 0.15) < 0.015
    assert abs(np.mean(cls == o.PAPER_NOISE) - 0.70) < 0.015
    for mk, mom, only in ((0, 0, o.PAPER_NOISE), (100, 0, o.PAPER_MAKER), (0, 100, o.PAPER_MOMENTUM)):
        p = dict(BASE, maker_pct=mk, mom_pct=mom)
        assert all(o.paper_class(p, gid) == only for gid in range(2000))


# --------------------------------------------------------------------------
# agent rules (Sec. III-C)
# --------------------------------------------------------------------------
def test_maker_alternates_and_quotes_the_rounded_half_spread():
    L = 64
    for D in (0, 1, 3):
        p = dict(BASE, maker_half_spread=D)
        for mid2 in range(0, 2 * L):
            for a, s in ((0, 0), (1, 0), (4, 7), (9, 12)):
                sd, tk, q = o.paper_order(p, L, 1000 + a, a, s, o.PAPER_MAKER, mid2, 1)
                assert sd == (a + s) % 2  # buys iff (a + s) mod 2 = 0
                x2 = mid2 + (2 * D if sd else -2 * D)  # 2 * (mid -/+ D)
                assert _nearest_even_ok(tk, x2, L), (mid2, D, sd, tk)
                assert 1 <= q <= p["qmax"]


def test_noise_orders():
    L, n = 128, 20000
    mid2 = 2 * 61 + 1  # mid 61.5
    sides, ticks, mkt = [], [], []
    for i in range(n):
        sd, tk, q = o.paper_order(BASE, L, i, i % 97, 5 + i % 3, o.PAPER_NOISE, mid2, 1)
        sides.append(sd)
        ticks.append(tk)
        mkt.append(tk == (0 if sd else L - 1))
    sides, ticks, mkt = np.array(sides), np.array(ticks), np.array(mkt)
    assert abs(sides.mean() - 0.5) < 0.015
    assert abs(mkt.mean() - 0.05) < 0.006  # P_mkt
    lim = ticks[~mkt]
    D = BASE["noise_halfwidth"]
    # round(mid + eta), eta in [-D, D]: ticks within [round(mid - D), round(mid + D)]
    assert lim.min() >= 57 and lim.max() <= 66
    # eta uniform: every interior tick carries 1/(2D) of the mass
    inner = [np.mean(lim == t) for t in range(58, 66)]
    assert max(abs(x - 1 / (2 * D)) for x in inner) < 0.015


def test_momentum_follows_the_mid_change():
    L = 128
    for mid2 in (100, 101, 130):
        for ret, want in ((1, 0), (-1, 1)):
            for i in range(300):
                sd, tk, q = o.paper_order(BASE, L, 77 + i, i, 3, o.PAPER_MOMENTUM, mid2, ret)
                assert sd == want
                if tk not in (0, L - 1):
                    assert _nearest_even_ok(tk, mid2 + (2 if sd == 0 else -2), L)
        sides = [o.paper_order(BASE, L, 5000 + i, i, 3, o.PAPER_MOMENTUM, mid2, 0)[0] for i in range(4000)]
        assert abs(np.mean(sides) - 0.5) < 0.03  # no change: random side


def test_quantity_uniform():
    q = np.array([o.paper_order(BASE, 64, i, i, 9, o.PAPER_NOISE, 64, 0)[2] for i in range(20000)])
    assert q.min() == 1 and q.max() == BASE["qmax"]
    for v in range(1, BASE["qmax"] + 1):
        assert abs(np.mean(q == v) - 1 / BASE["qmax"]) < 0.012


# --------------------------------------------------------------------------
# state retrieval and steps
# --------------------------------------------------------------------------
def test_mid_from_best_bid_and_ask():
    L = 32
    for bid_ticks, ask_ticks, last, want in (([3, 7], [12, 20], 9, 7 + 12), ([], [5], 9, 18), ([4], [], 6, 12),
                                             ([], [], 30, 60), ([0], [31], 2, 31)):
        bk = o.paper_init(900, L, 0)
        bk.sc.last = last
        for t in bid_ticks:
            bk.bid[t] = 5
        for t in ask_ticks:
            bk.ask[t] = 5
        o.paper_run(BASE, bk, 0, 1)  # no agents: the step only reads the mid
        assert bk.sc.mid2 == want


def _step_orders(params, market, L, A, s, mid2, ret):
    buy = np.zeros(L, np.int64)
    sell = np.zeros(L, np.int64)
    for a in range(A):
        gid = market * A + a
        sd, tk, q = o.paper_order(params, L, gid, a, s, o.paper_class(params, gid), mid2, ret)
        (sell if sd else buy)[tk] += q
    return buy, sell


def _brute_vstar(buy, sell):
    L = len(buy)
    return max(min(int(buy[p:].sum()), int(sell[:p + 1].sum())) for p in range(L))


def test_every_step_clears_the_steps_orders_and_rests_their_unfilled_part():
    for L, A, mom in ((16, 24, 15), (12, 40, 40), (32, 9, 0)):
        params = dict(BASE, mom_pct=mom)
        bk = o.paper_init(4, L, A)
        for s in range(40):
            bid0, ask0, last0, prev_mid2 = bk.bid.copy(), bk.ask.copy(), bk.sc.last, bk.sc.mid2
            bb = max([p for p in range(L) if bid0[p] > 0], default=-1)
            ba = min([p for p in range(L) if ask0[p] > 0], default=L)
            mid2 = bb + ba if bb >= 0 and ba < L else 2 * last0
            ret = (mid2 > prev_mid2) - (mid2 < prev_mid2)
            buy, sell = _step_orders(params, 4, L, A, s, mid2, ret)
            tp, tv = o.paper_run(params, bk, s, 1)
            v = _brute_vstar(buy, sell)
            assert tv[0] == v and bk.sc.mid2 == mid2
            nb, na = bk.bid.astype(np.int64), bk.ask.astype(np.int64)
            assert np.all((0 <= nb) & (nb <= buy)) and np.all((0 <= na) & (na <= sell))
            assert buy.sum() - nb.sum() == v and sell.sum() - na.sum() == v  # both sides trade V*
            # price priority: an unfilled buy at p means no buy below p traded (sells mirrored)
            for p in range(L):
                if nb[p] > 0:
                    assert np.array_equal(nb[:p], buy[:p])
                if na[p] > 0:
                    assert np.array_equal(na[p + 1:], sell[p + 1:])
            hb = max([p for p in range(L) if nb[p] > 0], default=-1)
            la = min([p for p in range(L) if na[p] > 0], default=L)
            assert hb < la  # the resting book is uncrossed
            if v > 0:
                p = tp[0]
                assert min(buy[p:].sum(), sell[:p + 1].sum()) == v  # p* executes V*
                assert all(min(buy[q:].sum(), sell[:q + 1].sum()) < v for q in range(p))  # lowest such tick
                assert bk.sc.last == p
            else:
                assert tp[0] == -1 and bk.sc.last == last0


def test_resume_equals_uninterrupted():
    L, A = 64, 50
    a = o.paper_init(7, L, A)
    ta = o.paper_run(BASE, a, 0, 60)
    b = o.paper_init(7, L, A)
    t1 = o.paper_run(BASE, b, 0, 23)
    t2 = o.paper_run(BASE, b, 23, 37)
    assert np.array_equal(ta[0], np.concatenate([t1[0], t2[0]]))
    assert np.array_equal(a.bid, b.bid) and np.array_equal(a.ask, b.ask)
    assert a.scalars() == b.scalars()


def test_makers_keep_a_noise_market_near_the_opening_price():
    # with quotes rounded half-up the makers would ratchet the price upward;
    # ties to even keep a noise/maker market centred (mean near L/2)
    params = dict(BASE, mom_pct=0, maker_pct=15)
    means = []
    for m in range(6):
        bk, tp, tv = o.paper_simulate(params, m, 128, 256, 300)
        means.append(tp[tp >= 0].mean())
    assert abs(np.mean(means) - 64) < 6


# ---- sliding window (Sec. III-A) ------------------------------------------------------------
def _drift_params(**over):
    p = dict(seed=11, noise_halfwidth=4, p_mkt_q32=0, qmax=10, maker_half_spread=1, mom_pct=70, maker_pct=15,
             tie_rule=0, window=0)
    p.update(over)
    return p


def _carried_price(tp, start):
    """Last clearing price after every step from a trace whose p* is -1 without trade."""
    out, last = np.empty(len(tp), np.int64), start
    for i, p in enumerate(tp):
        last = p if p >= 0 else last
        out[i] = last
    return out


@pytest.mark.parametrize("market,seed,mom,A", [(0, 7, 30, 200), (1, 7, 30, 200), (3, 5, 70, 200), (5, 7, 15, 200),
                                               (1, 7, 30, 5), (3, 7, 70, 3)])
def test_window_is_a_translation_of_a_large_grid(market, seed, mom, A):
    """Without marketable orders no order reaches the edge of a 64-tick window
    or of a 16384-tick grid, so the window must reproduce the large grid
    exactly, translated by the difference of the opening prices (8160, even).
    Momentum makes the price run away (up in market 1, down in market 0); the
    thin markets (A = 3, 5) trade on fewer than half of the steps and often
    leave a one-sided book, where the mid falls back to the last price."""
    S, Lw, Lb = 1500, 64, 16384
    off = Lb // 2 - Lw // 2
    bw = o.paper_init(market, Lw, A)
    tw_p, tw_v = o.paper_run(_drift_params(seed=seed, mom_pct=mom, window=1), bw, 0, S)
    bb = o.paper_init(market, Lb, A)
    tb_p, tb_v = o.paper_run(_drift_params(seed=seed, mom_pct=mom), bb, 0, S)
    price_b = _carried_price(tb_p, Lb // 2)
    assert 64 < price_b.min() and price_b.max() < Lb - 64          # the large grid never reached its edges
    assert price_b.max() - price_b.min() > Lw                      # wider than the window: it had to move
    assert np.array_equal(tw_v, tb_v)
    assert np.array_equal(tw_p.astype(np.int64), price_b - off)   # absolute last price after every step
    sw, sb = bw.scalars(), bb.scalars()
    assert sw["trades"] == sb["trades"] and sw["sum_v"] == sb["sum_v"]
    assert sw["sum_p"] == sb["sum_p"] - off * sb["trades"]
    assert sw["base"] + sw["last"] == sb["last"] - off and sb["base"] == 0
    # the resting book is the large grid's, seen through the window
    lo = sw["base"] + off
    assert np.array_equal(bw.bid, bb.bid[lo:lo + Lw]) and np.array_equal(bw.ask, bb.ask[lo:lo + Lw])
    assert bb.bid.sum() == bw.bid.sum() and bb.ask.sum() == bw.ask.sum()


def test_window_recentres_by_even_shifts_onto_the_centre():
    """Step by step: the window moves only when the mid is more than L/4 from
    the centre, always by an even number of ticks, and the moved mid lands
    within one tick of the centre; otherwise it stays."""
    L, A = 64, 150
    params = _drift_params(mom_pct=60, p_mkt_q32=214748365, window=1)  # P_mkt = 0.05
    bk = o.paper_init(2, L, A)
    moves = 0
    for s in range(1200):
        base0 = bk.scalars()["base"]
        # the mid this step starts from, in the current window
        bb = int(np.nonzero(bk.bid)[0].max()) if bk.bid.any() else -1
        ba = int(np.nonzero(bk.ask)[0].min()) if bk.ask.any() else L
        mid2 = bb + ba if (bb >= 0 and ba < L) else 2 * bk.scalars()["last"]
        o.paper_run(params, bk, s, 1)
        k = bk.scalars()["base"] - base0
        if abs(mid2 - L) > L // 2:
            assert k % 2 == 0 and k != 0
            assert bk.scalars()["mid2"] == mid2 - 2 * k and L <= mid2 - 2 * k < L + 4
            moves += 1
        else:
            assert k == 0 and bk.scalars()["mid2"] == mid2
    assert moves >= 5
