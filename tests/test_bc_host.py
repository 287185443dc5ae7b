"""Host logic of behaviour cloning: the canonical order of the records."""
import numpy as np
import torch

from paper_2606_21784_gb300 import bc


def test_canonical_order_is_lexicographic_and_order_free():
    rng = np.random.default_rng(3)
    r = rng.integers(-3, 4, size=(5000, 22)).astype(np.int32)
    r[100:200] = r[0]  # repeated records
    a = bc.canonical_order(torch.from_numpy(r))
    b = bc.canonical_order(torch.from_numpy(r[rng.permutation(len(r))]))
    assert torch.equal(a, b)
    want = r[np.lexsort(r.T[::-1])]  # first word most significant
    assert np.array_equal(a.numpy(), want)
