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
