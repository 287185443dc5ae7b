"""Tensor-core policy forward vs the fp64 oracle forward (max abs 2e-2 on logits)."""
import numpy as np
import pytest

import oracle as o
from paper_2606_21784_gb300 import kineticsim as ks

pytestmark = pytest.mark.gpu

LOGIT_TOL = 2e-2


def _params(rng, scale=0.25):
    W1 = rng.normal(0, scale, (64, 32))
    b1 = rng.normal(0, 0.1, 64)
    W2 = rng.normal(0, scale, (64, 64))
    b2 = rng.normal(0, 0.1, 64)
    W3 = rng.normal(0, scale, (37, 64))
    b3 = rng.normal(0, 0.1, 37)
    return W1, b1, W2, b2, W3, b3


def _features(rng, n):
    X = np.zeros((n, 32), np.float32)
    X[:, :8] = rng.integers(-8, 9, (n, 8)) / 8.0
    X[:, 8] = rng.integers(-300, 300, n) / 256.0
    X[:, 9] = rng.random(n) * 2
    X[:, 10:18] = rng.random((n, 8)) * 0.3
    return X


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 40000])
def test_tcgen05_forward_matches_fp64(n):
    import torch
    rng = np.random.default_rng(n)
    P = _params(rng)
    blob = ks.pack_mlp_params(*P)
    X = _features(rng, n)
    Z, err = ks.ks_mlp_forward(blob, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    w = o.mlp_pack(*ks.mlp_params_as_used(*P))
    ref = o.mlp_forward(w, X.astype(np.float64))
    got = Z.cpu().numpy().astype(np.float64)
    diff = np.abs(got - ref).max()
    assert diff <= LOGIT_TOL, diff


def test_tcgen05_forward_general_inputs():
    """All 32 inputs non-zero and of unit scale."""
    import torch
    rng = np.random.default_rng(7)
    P = _params(rng, 0.2)
    blob = ks.pack_mlp_params(*P)
    X = rng.normal(0, 1, (5000, 32)).astype(np.float32)
    Z, err = ks.ks_mlp_forward(blob, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = o.mlp_forward(o.mlp_pack(*ks.mlp_params_as_used(*P)), X.astype(np.float64))
    assert np.abs(Z.cpu().numpy() - ref).max() <= LOGIT_TOL
