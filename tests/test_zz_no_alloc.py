"""ks_step_n_noalloc: the batched launch with its scratch in the library's
static device array, for callers that cannot allocate device memory for the
kernel's work schedule and ticket counter (an allocator that is capped or
frozen, or a host framework that only hands out the buffers it owns).

Checks, through the C ABI, that two calls in a row give the oracle's state
and trace on every market, and exactly the state that two ks_step_n calls
give (the simulation is integer, so the tolerance of the other parity tests
is equality): for rule agents on the default plan, for a
1024-thread plan, and for the policy-capable kernel, on the default stream and
on a stream of its own.  Also checks the documented limits: a plain-mode
ensemble, too many markets and a capturing stream are refused.
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


def _policy_blob(seed=3, scale=0.3):
    rng = np.random.default_rng(seed)
    W1, b1 = rng.normal(0, scale, (64, 32)), rng.normal(0, 0.2, 64)
    W2, b2 = rng.normal(0, scale, (64, 64)), rng.normal(0, 0.2, 64)
    W3, b3 = rng.normal(0, scale, (37, 64)), rng.normal(0, 0.2, 37)
    b3[2] = -3.0
    b3[36] = np.log(30.0)
    return ks.pack_mlp_params(W1, b1, W2, b2, W3, b3)


def _pair(kind):
    """Two identical ensembles (reference, no-alloc) of the given kind."""
    if kind == "policy":
        M = 24
        L, A = wl.mixed_sizes(M, seed=9)
        A = np.minimum(A, 2048).astype(np.int32)
        w = wl.workload("mixed_32768", M=M)
        blob = _policy_blob()
        mk = lambda: ks.Ensemble(w, trace_markets=6, trace_steps=70, L=L, A=A, mlp_params=blob)  # noqa: E731
    else:
        M = 96
        L, A = wl.batched_sizes(M, seed=21)
        w = wl.workload("batched_20000", M=M)
        mk = lambda: ks.Ensemble(w, trace_markets=8, trace_steps=70, L=L, A=A)  # noqa: E731
    ref, got = mk(), mk()
    if kind == "plan1024":
        plan = (1024, [(2048, 16384, 1024, 16)])
        ref.set_batch_plan(*plan)
        got.set_batch_plan(*plan)
    return ref, got


def test_noalloc_matches_the_oracle():
    """Rule agents over two no-alloc calls, every market and its per-step trace
    against the oracle directly (not only through ks_step_n)."""
    import torch
    from helpers import compare_market, oracle_markets
    M = 40
    L, A = wl.batched_sizes(M, seed=23)
    w = wl.workload("batched_20000", M=M)
    ens = ks.Ensemble(w, trace_markets=M, trace_steps=70, L=L, A=A)
    assert ens.batch_info()["batched"] == 1
    assert _noalloc(ens, 45) == ks.KS_OK
    assert _noalloc(ens, 25) == ks.KS_OK
    torch.cuda.synchronize()
    assert ens.sync(timeout_ms=600_000) == ks.KS_OK
    gs = ens.read_state()
    for m, (mk, tp, tv) in oracle_markets(w["params"], range(M), L, A, 0, 70).items():
        compare_market(gs, ens, m, mk, tp, tv)


@pytest.mark.parametrize("kind,own_stream", [("rule", False), ("plan1024", True), ("policy", True)])
def test_noalloc_two_calls_match_ks_step_n(kind, own_stream):
    import torch
    ref, got = _pair(kind)
    assert ref.batch_info()["batched"] == 1 and got.batch_info()["batched"] == 1
    stream = torch.cuda.Stream() if own_stream else None
    torch.cuda.synchronize()
    ref.step(40, stream=stream)
    ref.step(30, stream=stream)
    assert _noalloc(got, 40, stream) == ks.KS_OK
    assert _noalloc(got, 30, stream) == ks.KS_OK
    torch.cuda.synchronize()
    assert ref.sync(timeout_ms=600_000) == ks.KS_OK
    assert got.sync(timeout_ms=600_000) == ks.KS_OK
    a, b = ref.read_state(), got.read_state()
    for f in a:
        assert np.array_equal(a[f], b[f]), (kind, f)
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


def test_noalloc_refuses_a_capturing_stream():
    import torch
    M = 8
    L, A = wl.batched_sizes(M, seed=4)
    ens = ks.Ensemble(wl.workload("batched_20000", M=M), L=L, A=A)
    assert _noalloc(ens, 2) == ks.KS_OK  # first call on the device outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        rc = _noalloc(ens, 2, s)
        g.capture_end()
    assert rc == ks.KS_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert ens.sync(timeout_ms=60_000) == ks.KS_OK
    assert int(ens.read_state()["step"][0]) == 2
