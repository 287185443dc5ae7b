"""Failure detection on the GPU, without faulting it.

- The host deadline of ks_sync: a wait shorter than the queued work returns
  KS_ERR_TIMEOUT and leaves the work running; a later wait returns KS_OK.
- The bounded device wait of the policy path: one warpgroup waits on an
  mbarrier that nothing arrives at (no tensor-core operation is issued, so
  none is in flight); the wait gives up within its wall-time limit, records
  the error bit ERR_MLP_WAIT (0x8) and returns; the next launch runs clean.
"""
import time

import numpy as np
import pytest

from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ERR_MLP_WAIT = 0x8


def test_sync_deadline_expires_then_the_run_completes():
    import torch
    w = wl.workload("plain_mix_8192", M=2048)
    ens = ks.Ensemble(w)
    ens.step(1)
    assert ens.sync(timeout_ms=120_000) == ks.KS_OK
    ens.step(1500)  # tens of milliseconds of device work
    assert ens.sync(timeout_ms=1) == ks.KS_ERR_TIMEOUT
    assert ens.sync(timeout_ms=600_000) == ks.KS_OK
    assert ks.ks_error_word(ens.handle) == 0
    assert int(ens.read_state(["step"])["step"][0]) == 1501
    torch.cuda.synchronize()


def test_bounded_device_wait_gives_up_and_the_next_launch_is_clean():
    import torch
    sink = torch.zeros(256 * 8 // 4, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ks.ks_probe(ks.KS_PROBE_WAIT_TIMEOUT, 1, 1, sink.data_ptr())
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = sink[:2].cpu().numpy()
    assert int(out[0]) == ERR_MLP_WAIT, out
    assert int(out[1]) == 1, out
    assert dt < 10.0, dt
    print(f"bounded wait gave up after {dt:.3f} s")
    # the context is intact: a policy ensemble runs clean afterwards
    rng = np.random.default_rng(0)
    P = [rng.normal(0, 0.3, s) for s in ((64, 32), 64, (64, 64), 64, (37, 64), 37)]
    blob = ks.pack_mlp_params(*P)
    ens = ks.Ensemble(wl.workload("learned_4096", M=4, L=256, A=512), mlp_params=blob)
    ens.step(10)
    assert ens.sync(timeout_ms=120_000) == ks.KS_OK
    assert ks.ks_error_word(ens.handle) == 0
    torch.cuda.synchronize()
