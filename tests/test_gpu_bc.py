"""Behaviour-cloning kernels vs the oracle, and what training gains."""
import numpy as np
import pytest

import oracle as o
from paper_2606_21784_gb300 import bc
from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_records():
    rec, w = bc.generate(n_pairs=400_000, markets=16, record_agents=64, steps=400)
    return rec, w


def _oracle_inputs(rec, A):
    r = rec.cpu().numpy()
    X = np.stack([o.mlp_features(x[:18], A) for x in r])
    return X, r[:, 18], r[:, 19], np.log(r[:, 20].astype(np.float64))


def test_bc_gradient_matches_fp64_oracle(small_records):
    import torch
    rec, w = small_records
    A = w["A"]
    sub = rec[:3000].contiguous()
    params = bc.init_params(3)
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ks.ks_bc_grad(params, sub, A, grad, loss, 1.0 / sub.shape[0])
    torch.cuda.synchronize()
    X, side, off, logq = _oracle_inputs(sub, A)
    l64, g64 = o.mlp_loss_grad(params.double().cpu().numpy(), X, side, off, logq)
    g = grad.double().cpu().numpy()
    assert abs(float(loss.item()) - l64) <= 1e-4 * max(1.0, abs(l64))
    assert np.abs(g - g64).max() <= 1e-4 * max(1.0, np.abs(g64).max())


def test_bc_gradient_is_deterministic_and_tail_safe(small_records):
    """The gradient is bit-identical across calls (fixed tile assignment and
    fixed-order sums); a ragged tail (n not a multiple of the 64-sample tile)
    matches the fp64 oracle too."""
    import torch
    rec, w = small_records
    A = w["A"]
    params = bc.init_params(4)
    outs = []
    for _ in range(3):
        grad = torch.zeros_like(params)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        ks.ks_bc_grad(params, rec[:50_000].contiguous(), A, grad, loss, 1.0 / 50_000)
        torch.cuda.synchronize()
        outs.append((grad.clone(), loss.clone()))
    for g, l in outs[1:]:
        assert torch.equal(g, outs[0][0]) and torch.equal(l, outs[0][1])
    sub = rec[:1001].contiguous()
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ks.ks_bc_grad(params, sub, A, grad, loss, 1.0 / 1001)
    torch.cuda.synchronize()
    X, side, off, logq = _oracle_inputs(sub, A)
    l64, g64 = o.mlp_loss_grad(params.double().cpu().numpy(), X, side, off, logq)
    assert abs(float(loss.item()) - l64) <= 1e-4 * max(1.0, abs(l64))
    assert np.abs(grad.double().cpu().numpy() - g64).max() <= 1e-4 * max(1.0, np.abs(g64).max())


def test_workspace_too_small_is_refused():
    import ctypes

    import torch
    params = bc.init_params(0)
    rec = torch.zeros((1000, ks.KS_RECORD_WORDS), dtype=torch.int32, device="cuda")
    rec[:, 20] = 1
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    need = ks.ks_bc_workspace_size(1000)
    assert need > 0
    ws = torch.empty(need - 4, dtype=torch.uint8, device="cuda")
    rc = ks.load().ks_bc_grad(params.data_ptr(), rec.data_ptr(), 1000, 64, grad.data_ptr(), loss.data_ptr(),
                              ctypes.c_float(1.0), ws.data_ptr(), ws.numel(), None)
    assert rc == ks.KS_ERR_WORKSPACE_TOO_SMALL
    torch.cuda.synchronize()


def test_training_is_reproducible(small_records):
    """Two training runs from the same seed give the same network bit for bit."""
    import torch
    rec, w = small_records
    p1, h1, _ = bc.train(rec[:120_000], w["A"], epochs=1, batch=4096, lr=3e-3, seed=5)
    p2, h2, _ = bc.train(rec[:120_000], w["A"], epochs=1, batch=4096, lr=3e-3, seed=5)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
    assert h1 == h2


def test_generation_is_reproducible():
    """The records (and so the network) follow from the arguments alone: the
    kernels append in completion order; a full capacity is rerun; a subset
    is drawn by the seed."""
    import torch
    kw = dict(n_pairs=10_000, markets=8, record_agents=64, steps=300)
    a, _ = bc.generate(**kw)
    b, _ = bc.generate(**kw)
    assert a.shape == (10_000, 22)
    assert torch.equal(a, b)
    c, _ = bc.generate(**dict(kw, n_pairs=10**6))  # every record, no subset
    assert c.shape[0] > 10_000
    assert torch.equal(c, bc.canonical_order(c))
    d, _ = bc.generate(**dict(kw, n_pairs=10**6))
    assert torch.equal(c, d)


def test_adam_step_matches_fp64_oracle():
    import torch
    rng = np.random.default_rng(0)
    n = ks.KS_MLP_NPARAM
    w0 = rng.normal(size=n)
    g0 = rng.normal(size=n)
    m0 = rng.normal(size=n) * 0.1
    v0 = rng.random(n) * 0.1
    P = torch.tensor(w0, dtype=torch.float32, device="cuda")
    G = torch.tensor(g0, dtype=torch.float32, device="cuda")
    M = torch.tensor(m0, dtype=torch.float32, device="cuda")
    V = torch.tensor(v0, dtype=torch.float32, device="cuda")
    ks.ks_adam_step(P, G, M, V, 3, 1e-2)
    torch.cuda.synchronize()
    w, m, v = (x.astype(np.float64).copy() for x in (np.float32(w0), np.float32(m0), np.float32(v0)))
    o.adam_step(w, np.float32(g0).astype(np.float64), m, v, 3, 1e-2)
    assert np.allclose(P.cpu().numpy(), w, atol=1e-5)
    assert np.allclose(M.cpu().numpy(), m, atol=1e-6) and np.allclose(V.cpu().numpy(), v, atol=1e-6)
    assert float(G.abs().max()) == 0.0


def test_export_matches_host_packing():
    import torch
    p = bc.init_params(5)
    blob = bc.export(p)
    parts = o.mlp_unpack(p.double().cpu().numpy())
    ref = ks.pack_mlp_params(*parts)
    torch.cuda.synchronize()
    assert torch.equal(blob.cpu(), ref.cpu())


def test_training_gains_over_untrained_and_marginal_policies(small_records):
    """Held-out loss and action agreement: trained beats both the untrained
    network and the best input-independent policy; the trained policy's
    markets are closer to the rule-based markets than the untrained one's."""
    rec, w = small_records
    A = w["A"]
    params, hist, val = bc.train(rec, A, epochs=3, batch=8192, lr=3e-3, val_frac=0.1)
    l_trained = bc.evaluate(params, val, A)
    l_init = bc.evaluate(bc.init_params(0), val, A)
    l_marg = bc.evaluate(bc.marginal_params(rec), val, A)
    print(f"held-out loss: trained {l_trained:.4f}  marginal {l_marg:.4f}  untrained {l_init:.4f}")
    assert l_trained < l_marg < l_init
    m_tr = bc.action_match(bc.export(params), val, A)
    m_mg = bc.action_match(bc.export(bc.marginal_params(rec)), val, A)
    print("action match trained", m_tr, "marginal", m_mg)
    assert m_tr["error_word"] == 0
    assert m_tr["side"] > m_mg["side"] and m_tr["offset"] >= m_mg["offset"]

    def market_stats(blob, mlp_pct):
        import torch
        ww = wl.workload("learned_4096", M=64, L=1024, A=1024, mlp_pct=mlp_pct, seed=11)
        ens = ks.Ensemble(ww, trace_markets=64, trace_steps=300, mlp_params=blob)
        ens.step(300)
        torch.cuda.synchronize()
        tr = ens.read_state()["trace"]
        p, v = tr[:, 100:, 0].astype(float), tr[:, 100:, 1].astype(float)
        px = np.where(p < 0, np.nan, p)
        ret = np.nanstd(np.diff(px, axis=1))
        return np.array([v.mean() / 1024, ret])

    rule = market_stats(bc.export(params), 0)
    trained = market_stats(bc.export(params), 100)
    untrained = market_stats(bc.export(bc.init_params(0)), 100)
    print("market stats (volume/agent, return std): rule", rule, "trained", trained, "untrained", untrained)
    d_tr = np.abs((trained - rule) / rule).sum()
    d_un = np.abs((untrained - rule) / rule).sum()
    assert d_tr < d_un
