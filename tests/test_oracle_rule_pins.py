"""Pins of the oracle's rule decisions (readings R7, R10-R12) from draw words
chosen at the boundaries where a decision changes:

- the quantity is the paper's q = 1 + floor(u q_max) with u = w3 / 2^32
  (Sec. III-C): the smallest word giving q = k + 1 is ceil(k 2^32 / q_max);
- a zero-intelligence side is the coin (buy iff w1 < 2^31), its tick
  last - D + floor(w2 (2D + 1) / 2^32), clamped to the grid;
- momentum buys above the last tick after a rise of the lookback return and
  sells below it after a fall (the coin when flat); mean reversion trades
  toward the fundamental (the coin at it); both move o = floor(w2 (omax + 1)
  / 2^32) ticks through the last tick.
Every boundary is computed here with exact integer arithmetic."""
import pytest

import oracle as o

ZI, MOM, MR = 0, 1, 2
BUY, SELL = 0, 1
TWO32 = 1 << 32


def _params(**over):
    from paper_2606_21784_gb300 import workloads as wl
    p = dict(wl.workload("plain_mix_8192")["params"])
    p.update(over)
    return p


def _first_word(k, n):
    """Smallest 32-bit w with floor(w n / 2^32) >= k."""
    return -(-k * TWO32 // n)


def _dec(p, atype, w, last=500, hist=None, fund=500, L=1024):
    return o.rule_decision(p, L, atype, last, hist or [last] * 9, fund, w)


@pytest.mark.parametrize("qmax", [1, 7, 10, 100, 255])
@pytest.mark.parametrize("atype", [ZI, MOM, MR])
def test_quantity_is_one_plus_floor_u_qmax(atype, qmax):
    p = _params(zi_qmax=qmax, rb_qmax=qmax)
    assert _dec(p, atype, [0, 0, 0, 0])[2] == 1
    assert _dec(p, atype, [0, 0, 0, TWO32 - 1])[2] == qmax
    for k in range(1, qmax):
        w = _first_word(k, qmax)
        assert _dec(p, atype, [0, 0, 0, w])[2] == k + 1, (k, w)
        assert _dec(p, atype, [0, 0, 0, w - 1])[2] == k, (k, w)


def test_zero_intelligence_side_is_the_coin():
    p = _params()
    assert _dec(p, ZI, [0, (1 << 31) - 1, 0, 0])[0] == BUY
    assert _dec(p, ZI, [0, 1 << 31, 0, 0])[0] == SELL
    assert _dec(p, ZI, [0, TWO32 - 1, 0, 0])[0] == SELL


@pytest.mark.parametrize("D", [0, 1, 16, 32])
def test_zero_intelligence_tick_boundaries(D):
    p = _params(zi_offset=D)
    n = 2 * D + 1
    last = 500
    assert _dec(p, ZI, [0, 0, 0, 0], last=last)[1] == last - D
    assert _dec(p, ZI, [0, 0, TWO32 - 1, 0], last=last)[1] == last + D
    for j in range(1, n):
        w = _first_word(j, n)
        assert _dec(p, ZI, [0, 0, w, 0], last=last)[1] == last - D + j
        assert _dec(p, ZI, [0, 0, w - 1, 0], last=last)[1] == last - D + j - 1


def test_ticks_clamp_to_the_grid():
    p = _params(zi_offset=32, mom_offset_max=8)
    assert _dec(p, ZI, [0, 0, 0, 0], last=3, L=64)[1] == 0
    assert _dec(p, ZI, [0, 0, TWO32 - 1, 0], last=60, L=64)[1] == 63
    rise = [62] + [50] * 8
    assert _dec(p, MOM, [0, 0, TWO32 - 1, 0], last=62, hist=rise, L=64)[1] == 63


@pytest.mark.parametrize("lb", [1, 4, 8])
def test_momentum_follows_the_lookback_return(lb):
    p = _params(mom_lookback=lb, mom_offset_max=8)
    last = 400
    w_far = _first_word(8, 9)  # offset 8 (the largest)
    rise = [last] * 9
    rise[lb] = last - 3
    fall = [last] * 9
    fall[lb] = last + 3
    for coin in (0, TWO32 - 1):  # the side does not depend on the coin
        assert _dec(p, MOM, [0, coin, w_far, 0], last=last, hist=rise)[:2] == (BUY, last + 8)
        assert _dec(p, MOM, [0, coin, w_far, 0], last=last, hist=fall)[:2] == (SELL, last - 8)
    other = [last] * 9
    other[lb % 8 + 1] = last - 3  # a change at another lag does not count
    if lb % 8 + 1 != lb:
        assert _dec(p, MOM, [0, 0, 0, 0], last=last, hist=other)[0] == BUY  # flat return: the coin (buy)
        assert _dec(p, MOM, [0, TWO32 - 1, 0, 0], last=last, hist=other)[0] == SELL
    for j in range(1, 9):
        w = _first_word(j, 9)
        assert _dec(p, MOM, [0, 0, w, 0], last=last, hist=rise)[1] == last + j
        assert _dec(p, MOM, [0, 0, w - 1, 0], last=last, hist=rise)[1] == last + j - 1


def test_mean_reversion_trades_toward_the_fundamental():
    p = _params(mr_offset_max=8)
    w5 = _first_word(5, 9)
    for coin in (0, TWO32 - 1):
        assert _dec(p, MR, [0, coin, w5, 0], last=300, fund=450)[:2] == (BUY, 305)
        assert _dec(p, MR, [0, coin, w5, 0], last=600, fund=450)[:2] == (SELL, 595)
    assert _dec(p, MR, [0, 0, w5, 0], last=450, fund=450)[:2] == (BUY, 455)
    assert _dec(p, MR, [0, TWO32 - 1, w5, 0], last=450, fund=450)[:2] == (SELL, 445)


def test_each_class_takes_its_own_quantity_range():
    """Zero intelligence draws 1..zi_qmax, momentum and mean reversion 1..rb_qmax."""
    p = _params(zi_qmax=10, rb_qmax=100)
    top = TWO32 - 1
    assert _dec(p, ZI, [0, 0, 0, top])[2] == 10
    assert _dec(p, MOM, [0, 0, 0, top])[2] == 100
    assert _dec(p, MR, [0, 0, 0, top])[2] == 100


def test_classes_policy_flags_and_fundamental_from_their_streams():
    """Agent a of market m takes its class from the percentile floor(w0 100 / 2^32)
    of Philox counter (0, a, m, 1) against the cumulative mix (zero intelligence
    below mix[0], momentum below mix[0] + mix[1]) and its policy flag from the
    percentile of w1 against mlp_pct; the fundamental is L/4 + floor(w0 (L/2 + 1)
    / 2^32) of counter (0, 0, m, 2).  Checked with the generator the Philox
    known-answer vectors pin."""
    p = _params(mix_pct=(55, 25, 20), mlp_pct=30)
    seed = int(p["seed"])
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for m, L, A in ((0, 1024, 400), (77, 129, 300)):
        mk = o.init_market(p, m, L, A)
        for a in range(A):
            w = o.philox4x32_10((0, a, m, 1), key)
            pct = int(w[0]) * 100 >> 32
            want = ZI if pct < 55 else (MOM if pct < 80 else MR)
            assert mk.atype[a] == want, (m, a)
            assert mk.mlp[a] == (1 if (int(w[1]) * 100 >> 32) < 30 else 0), (m, a)
        wf = o.philox4x32_10((0, 0, m, 2), key)
        assert mk.sc.fund == L // 4 + (int(wf[0]) * (L // 2 + 1) >> 32)
        assert mk.sc.last == L // 2 and list(mk.sc.hist) == [L // 2] * 9
