"""Pins of the oracle's fp64 policy network, loss, gradient and sampling.

Expected values come from closed forms (a permutation network whose logits
are its inputs, the loss at zero weights) and from finite differences of the
oracle's own loss (which checks the analytic backward against the forward).
"""
import math

import numpy as np
import pytest

import oracle as o


def _random_params(rng, scale=0.3):
    return rng.normal(0, scale, o.mlp_nparam())


def test_permutation_network_returns_its_input():
    """W1 routes x[pi(i)] and -x[pi(i)] through ReLU pairs, W2 is the identity,
    W3 recombines relu(x) - relu(-x) = x; so z[j] = x[j] + b3[j] for j < 32."""
    rng = np.random.default_rng(1)
    pi = rng.permutation(32)
    W1 = np.zeros((64, 32))
    for i in range(32):
        W1[i, pi[i]] = 1.0
        W1[32 + i, pi[i]] = -1.0
    W2 = np.eye(64)
    W3 = np.zeros((37, 64))
    for i in range(32):
        W3[pi[i], i] = 1.0
        W3[pi[i], 32 + i] = -1.0
    b3 = rng.normal(size=37)
    w = o.mlp_pack(W1, np.zeros(64), W2, np.zeros(64), W3, b3)
    X = rng.normal(size=(50, 32))
    Z = o.mlp_forward(w, X)
    assert np.allclose(Z[:, :32], X + b3[:32], atol=1e-12)
    assert np.allclose(Z[:, 32:], b3[32:], atol=1e-12)


def test_loss_at_zero_weights_closed_form():
    rng = np.random.default_rng(2)
    n = 40
    X = rng.normal(size=(n, 32))
    side = rng.integers(0, 3, n)
    off = rng.integers(0, 33, n)
    logq = np.log(rng.integers(1, 101, n).astype(float))
    loss, g = o.mlp_loss_grad(np.zeros(o.mlp_nparam()), X, side, off, logq)
    assert abs(loss - (math.log(3) + math.log(33) + np.mean(logq ** 2))) < 1e-12


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    n = 16
    w = _random_params(rng)
    X = rng.normal(size=(n, 32))
    side = rng.integers(0, 3, n)
    off = rng.integers(0, 33, n)
    logq = np.log(rng.integers(1, 101, n).astype(float))
    _, g = o.mlp_loss_grad(w, X, side, off, logq)
    idx = rng.choice(o.mlp_nparam(), 120, replace=False)
    h = 1e-6
    for i in idx:
        wp = w.copy(); wp[i] += h
        wm = w.copy(); wm[i] -= h
        lp, _ = o.mlp_loss_grad(wp, X, side, off, logq)
        lm, _ = o.mlp_loss_grad(wm, X, side, off, logq)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_sampling_inverse_cdf():
    # a certain class is always drawn
    z = np.full(37, -1000.0)
    z[1] = 0.0
    z[3 + 20] = 0.0
    z[36] = math.log(37.0)
    for w0 in (0, 1 << 31, 0xFFFFFFFF):
        sd, oi, q = o.mlp_action(z, [w0, w0, 0, 0], 100)
        assert (sd, oi, q) == (1, 20, 37)
    # equal logits: the draw is floor(n u) away from the class boundaries
    z = np.zeros(37)
    rng = np.random.default_rng(4)
    for _ in range(200):
        w0, w1 = (int(x) for x in rng.integers(0, 2 ** 32, 2))
        u0, u1 = w0 / 2 ** 32, w1 / 2 ** 32
        if min(abs(u0 * 3 - round(u0 * 3)), abs(u1 * 33 - round(u1 * 33))) < 1e-9:
            continue
        sd, oi, q = o.mlp_action(z, [w0, w1, 0, 0], 100)
        assert sd == int(u0 * 3) and oi == int(u1 * 33) and q == 1


@pytest.mark.parametrize("y,qmax,want", [(math.log(2.5), 100, 3), (math.log(2.49), 100, 2), (10.0, 100, 100),
                                         (-5.0, 100, 1), (math.log(200.0), 255, 200)])
def test_quantity_rounding_and_clamps(y, qmax, want):
    z = np.zeros(37)
    z[36] = y
    assert o.mlp_action(z, [0, 0, 0, 0], qmax)[2] == want


def test_feature_normalisation():
    raw = np.arange(1, 19, dtype=np.int32)
    x = o.mlp_features(raw, 2048)
    assert np.allclose(x[:8], raw[:8] / 8.0)
    assert x[8] == raw[8] / 256.0
    assert x[9] == raw[9] / (8.0 * 2048)
    assert np.allclose(x[10:18], raw[10:18] / (4.0 * 2048))
    assert np.all(x[18:] == 0)


def test_recorded_rule_decisions_describe_the_new_orders():
    """Records of rule decisions carry the features and the action of the order placed."""
    from paper_2606_21784_gb300 import workloads as wl
    params = dict(wl.workload("plain_mix_8192")["params"], cancel_thresh_q32=0)
    mk = o.init_market(params, 0, 256, 64)
    stats = {}
    for s in range(30):
        before = mk.qty.copy()
        last = mk.last
        hist = mk.hist.copy()
        o.run_market(params, mk, s, 1, rec_agents=64, rec_cap=1000, stats=stats)
        rec = stats["records"]
        new = np.nonzero(before == 0)[0]
        assert len(rec) == len(new)
        for r, a in zip(rec, new):
            assert list(r[:8]) == [int(hist[j] - hist[j + 1]) for j in range(8)]
            assert r[21] == mk.atype[a]
            # a recorded order that rested is still the agent's working order
            if mk.qty[a] > 0 and mk.qty[a] == r[20]:
                assert r[18] == mk.side[a]
                toward = (last - mk.tick[a]) if mk.side[a] == 1 else (mk.tick[a] - last)
                assert r[19] == int(np.clip(toward, -16, 16)) + 16
            assert r[18] in (0, 1) and 0 <= r[19] <= 32 and 1 <= r[20] <= 100
            if r[21] != o.ZI:  # momentum / mean-reversion orders go through the price
                assert 16 <= r[19] <= 24


# ---------------------------------------------------------------------------
# Raw policy features of a hand-built book (the market-level part of the
# policy input: returns, last V*, resting depth around the last tick, all
# taken at the start of the step, before cancellations)
# ---------------------------------------------------------------------------
def _carry_params():
    from paper_2606_21784_gb300 import workloads as wl
    return dict(wl.workload("plain_mix_8192")["params"])


def _cancelled_at(params, m, s, agents):
    """Agents whose step-s cancellation word is below the threshold (counter (s, a, m, 0))."""
    seed = int(params["seed"])
    key = (seed & 0xFFFFFFFF, seed >> 32)
    return [a for a in agents if int(o.philox4x32_10((s, a, m, 0), key)[0]) < int(params["cancel_thresh_q32"])]


def _records_of_hand_book(L, last, hist, last_v, orders, A=48, s=5, m=3):
    """Runs one step of a market whose resting book is `orders` ({agent:
    (side, tick, qty)}); returns the records of the deciding agents in agent
    order, the deciding agents, and their inventories."""
    params = _carry_params()
    mk = o.init_market(params, m, L, A)
    mk.sc.last = last
    for j in range(9):
        mk.sc.hist[j] = hist[j]
    mk.sc.last_v = last_v
    mk.inv[:] = 1000 + 7 * np.arange(A)
    mk.qty[:] = 0
    for a, (sd, tk, q) in orders.items():
        mk.side[a], mk.tick[a], mk.qty[a] = sd, tk, q
    inv0 = mk.inv.copy()
    cancelled = _cancelled_at(params, m, s, sorted(orders))
    deciders = sorted(set(range(A)) - set(orders) | set(cancelled))
    stats = {}
    o.run_market(params, mk, s, 1, rec_agents=A, rec_cap=4 * A, stats=stats)
    return stats["records"], deciders, inv0, cancelled


def _check_features(rec, deciders, inv0, hist, last_v, asks, bids):
    assert len(rec) == len(deciders)
    for r, a in zip(rec, deciders):
        assert list(r[:8]) == [hist[j] - hist[j + 1] for j in range(8)]
        assert r[8] == inv0[a]
        assert r[9] == last_v
        assert list(r[10:14]) == asks, (list(r[10:14]), asks)
        assert list(r[14:18]) == bids, (list(r[14:18]), bids)


def test_raw_features_of_a_hand_built_book():
    """Last tick 30 of 64.  Expected depth, written out by hand:
    asks at 31..34 = (5 + 7, 10, 4, 0); bids at 29..26 = (6, 0, 2 + 1, 8).
    The 10 at tick 32 is an order that this step's cancellation removes (the
    depth is taken before cancellations).  Orders at the last tick, beyond 4
    ticks, and on the other side of the book (a buy at 32, a sell at 28) do
    not count."""
    L, last, last_v = 64, 30, 123
    hist = [30, 27, 33, 33, 20, 25, 31, 31, 40]
    params = _carry_params()
    cands = _cancelled_at(params, 3, 5, range(48))
    assert cands, "no agent cancels at this step; pick another step"
    c = cands[0]
    free = [a for a in range(48) if a not in cands]
    BUY, SELL = 0, 1
    book = [(SELL, 31, 5), (SELL, 31, 7), (SELL, 33, 4), (SELL, 35, 9), (BUY, 29, 6), (SELL, 28, 13),
            (BUY, 32, 11), (BUY, 27, 2), (BUY, 27, 1), (BUY, 26, 8), (BUY, 25, 3), (SELL, 30, 2), (BUY, 30, 4)]
    orders = {a: o_ for a, o_ in zip(free, book)}
    orders[c] = (SELL, 32, 10)
    rec, dec, inv0, cancelled = _records_of_hand_book(L, last, hist, last_v, orders)
    assert c in cancelled
    _check_features(rec, dec, inv0, hist, last_v, asks=[12, 10, 4, 0], bids=[6, 0, 3, 8])


@pytest.mark.parametrize("where", ["low", "high"])
def test_raw_features_at_the_grid_edges(where):
    """Ticks beyond the grid hold no depth: last tick 1 (bids only at tick 0)
    and last tick L-2 (asks only at tick L-1)."""
    L, last_v = 64, 7
    BUY, SELL = 0, 1
    if where == "low":
        last = 1
        book = [(BUY, 0, 5), (SELL, 0, 9), (SELL, 2, 3), (SELL, 5, 7), (SELL, 6, 1)]
        asks, bids = [3, 0, 0, 7], [5, 0, 0, 0]
    else:
        last = L - 2
        book = [(SELL, L - 1, 4), (BUY, L - 1, 9), (BUY, L - 3, 2), (BUY, L - 6, 6), (BUY, L - 7, 1)]
        asks, bids = [4, 0, 0, 0], [2, 0, 0, 6]
    hist = [last] * 9
    params = _carry_params()
    stay = [a for a in range(48) if a not in _cancelled_at(params, 3, 5, range(48))]
    orders = {a: o_ for a, o_ in zip(stay, book)}
    rec, dec, inv0, _ = _records_of_hand_book(L, last, hist, last_v, orders)
    _check_features(rec, dec, inv0, hist, last_v, asks, bids)


# ---------------------------------------------------------------------------
# Adam (Kingma and Ba, ICLR 2015): bias-corrected steps computed by hand
# ---------------------------------------------------------------------------
def _adam_run(grads, lr, b1, b2, eps, w0):
    w = np.array(w0, np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    out = []
    for t, g in enumerate(grads, start=1):
        o.adam_step(w, np.array(g, np.float64), m, v, t, lr, b1, b2, eps)
        out.append((w.copy(), m.copy(), v.copy()))
    return out


def test_adam_two_steps_by_hand():
    """b1 = 1/2, b2 = 3/4, lr = 0.1, eps = 0, gradients g1 = (1, -2, 1/2) and
    g2 = (3, 2, -1/2).  Step 1: m = g1/2, v = g1^2/4 and the bias-corrected
    step is lr * sign(g1).  Step 2: m = g1/4 + g2/2 = (7/4, 1/2, -1/8),
    v = 3 g1^2/16 + g2^2/4 = (39/16, 7/4, 7/64); corrected by 1 - b1^2 = 3/4
    and 1 - b2^2 = 7/16: m_hat = (7/3, 2/3, -1/6), v_hat = (39/7, 4, 1/4)."""
    w0 = [0.5, -1.0, 2.0]
    (w1, m1, v1), (w2, m2, v2) = _adam_run([[1, -2, 0.5], [3, 2, -0.5]], 0.1, 0.5, 0.75, 0.0, w0)
    assert np.allclose(m1, [0.5, -1.0, 0.25], rtol=0, atol=1e-15)
    assert np.allclose(v1, [0.25, 1.0, 0.0625], rtol=0, atol=1e-15)
    assert np.allclose(w1, [0.4, -0.9, 1.9], rtol=0, atol=1e-15)
    assert np.allclose(m2, [7 / 4, 1 / 2, -1 / 8], rtol=0, atol=1e-15)
    assert np.allclose(v2, [39 / 16, 7 / 4, 7 / 64], rtol=0, atol=1e-15)
    step2 = [0.1 * (7 / 3) / math.sqrt(39 / 7), 0.1 * (2 / 3) / 2.0, 0.1 * (-1 / 6) / 0.5]
    assert np.allclose(w2, np.array([0.4, -0.9, 1.9]) - step2, rtol=0, atol=1e-14)


def test_adam_constant_gradient_steps_are_constant():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2 at every t, so every step is lr * g / (|g| + eps); eps = 1/4 here,
    large enough that it must sit outside the square root."""
    g = [2.0, -0.5, 1e-3]
    lr, eps = 0.01, 0.25
    runs = _adam_run([g] * 6, lr, 0.9, 0.999, eps, [0.0, 0.0, 0.0])
    step = np.array([lr * x / (abs(x) + eps) for x in g])
    prev = np.zeros(3)
    for t, (w, _, _) in enumerate(runs, start=1):
        assert np.allclose(prev - w, step, rtol=1e-12, atol=0), t
        prev = w
