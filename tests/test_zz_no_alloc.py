"""ks_step_n_noalloc: the batched launch with its scratch in the library's
static device array, for callers that cannot allocate device memory for the
kernel's work schedule and ticket counter.

Checks, through the C ABI, that two calls in a row give exactly the state that
two ks_step_n calls give (the simulation is integer, so the tolerance of the
other parity tests is equality), and that the documented limits are enforced.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _noalloc(ens, n_steps, stream=None):
    lib = ks.load()
    f = lib.ks_step_n_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f(ens.handle, int(n_steps), ks._stream_ptr(stream))


def test_noalloc_two_calls_match_ks_step_n():
    import torch
    M = 96
    L, A = wl.batched_sizes(M, seed=21)
    w = wl.workload("batched_20000", M=M)
    ref = ks.Ensemble(w, trace_markets=8, trace_steps=70, L=L, A=A)
    got = ks.Ensemble(w, trace_markets=8, trace_steps=70, L=L, A=A)
    assert ref.batch_info()["batched"] == 1 and got.batch_info()["batched"] == 1
    ref.step(40)
    ref.step(30)
    assert _noalloc(got, 40) == ks.KS_OK
    assert _noalloc(got, 30) == ks.KS_OK
    torch.cuda.synchronize()
    assert got.sync(timeout_ms=600_000) == ks.KS_OK
    a, b = ref.read_state(), got.read_state()
    for f in a:
        assert np.array_equal(a[f], b[f]), f
    assert int(b["step"][0]) == 70


def test_noalloc_limits():
    import torch
    # a plain-mode ensemble does not run the batched kernel
    plain = ks.Ensemble(wl.workload("plain_mix_8192", M=4))
    assert plain.batch_info()["batched"] == 0
    assert _noalloc(plain, 5) == ks.KS_ERR_INVALID_ARG
    # more markets than the static array holds
    M = 32769
    big = ks.Ensemble(wl.workload("batched_20000", M=M), L=np.full(M, 2, np.int32),
                      A=np.where(np.arange(M) % 2 == 0, 1, 2).astype(np.int32))
    assert big.batch_info()["batched"] == 1
    assert _noalloc(big, 1) == ks.KS_ERR_UNSUPPORTED
    torch.cuda.synchronize()
