"""GPU <-> oracle parity of the persistent kernel, bit-exact, through the C ABI."""
import numpy as np
import pytest

import oracle as o
from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

from helpers import compare_market, oracle_markets

pytestmark = pytest.mark.gpu


def _run_gpu(w, steps, trace_markets=0, launch=None, chunks=None, L=None, A=None):
    import torch
    ens = ks.Ensemble(w, trace_markets=trace_markets, trace_steps=steps if trace_markets else 0, L=L, A=A)
    if launch:
        ens.set_launch(**launch)
    for c in (chunks or [steps]):
        ens.step(c)
    assert ens.sync(timeout_ms=600_000) == ks.KS_OK
    torch.cuda.synchronize()
    return ens, ens.read_state()


def test_plain_zi_every_market_every_step():
    """64 markets, L=256, A=256, 1000 steps, discard mode: every market and step."""
    w = wl.workload("plain_zi_64")
    ens, gs = _run_gpu(w, w["S"], trace_markets=w["M"])
    L, A = ens.L, ens.A
    ref = oracle_markets(w["params"], range(w["M"]), L, A, 0, w["S"])
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp, tv)
    assert int(gs["step"][0]) == w["S"]


def test_plain_mix_reduced_every_market():
    """Carried book, 60/20/20 agent mix, L=1024, A=4096, 24 markets x 150 steps."""
    w = wl.workload("plain_mix_8192", M=24)
    steps = 150
    ens, gs = _run_gpu(w, steps, trace_markets=w["M"])
    ref = oracle_markets(w["params"], range(w["M"]), ens.L, ens.A, 0, steps)
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp, tv)


@pytest.mark.parametrize("launch", [
    dict(threads=256, agents_per_thread=16),
    dict(threads=512, agents_per_thread=8),
    dict(threads=1024, agents_per_thread=4),
    dict(threads=512, agents_per_thread=8, aggregate=1),
    dict(threads=256, agents_per_thread=16, ctas_per_sm=1, aggregate=1),
    dict(threads=512, agents_per_thread=8, reg_cap=3),
    dict(threads=1024, agents_per_thread=4, reg_cap=3),
    # the carried-book kernels (full shapes in the 128-register class)
    dict(threads=256, agents_per_thread=16, reg_cap=1),
    dict(threads=512, agents_per_thread=8, reg_cap=1),
])
def test_launch_shape_invariance(launch):
    """Any launch shape gives the same state (races in aggregation or allocation would differ)."""
    w = wl.workload("plain_mix_8192", M=40)
    steps = 60
    ens, gs = _run_gpu(w, steps, trace_markets=4, launch=launch)
    ref = oracle_markets(w["params"], range(w["M"]), ens.L, ens.A, 0, steps)
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp if m < 4 else None, tv if m < 4 else None)


def test_split_calls_equal_one_call():
    w = wl.workload("plain_mix_8192", M=16)
    _, a = _run_gpu(w, 90, trace_markets=16)
    _, b = _run_gpu(w, 90, trace_markets=16, chunks=[1, 29, 60])
    for f in a:
        assert np.array_equal(a[f], b[f]), f


def test_checkpoint_resume():
    """read_state -> new ensemble -> write_state -> continue equals an uninterrupted run."""
    import torch
    w = wl.workload("plain_mix_8192", M=12)
    _, full = _run_gpu(w, 80)
    ens1, mid = _run_gpu(w, 35)
    ens2 = ks.Ensemble(w)
    ens2.write_state({k: v for k, v in mid.items() if k != "trace"})
    ens2.step(45)
    torch.cuda.synchronize()
    res = ens2.read_state()
    for f in full:
        if f != "trace":
            assert np.array_equal(full[f], res[f]), f


def test_edge_shapes_ragged_and_tiny():
    """Ragged agent counts, non-power-of-two grids, L=2, A=1 and A=0 markets in one ensemble."""
    Ls = np.array([2, 3, 100, 1000, 130, 64, 2048, 7, 256, 4096], np.int32)
    As = np.array([1, 5, 77, 999, 0, 3000, 513, 1, 16384, 700], np.int32)
    w = wl.workload("plain_mix_8192", M=len(Ls))
    steps = 40
    ens, gs = _run_gpu(w, steps, trace_markets=len(Ls), L=Ls, A=As)
    ref = oracle_markets(w["params"], range(len(Ls)), Ls, As, 0, steps)
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp, tv)


def test_tie_rule_min_imbalance():
    w = wl.workload("plain_zi_64", M=16, tie_rule=1)
    ens, gs = _run_gpu(w, 200, trace_markets=16)
    ref = oracle_markets(w["params"], range(16), ens.L, ens.A, 0, 200)
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp, tv)


def test_graph_capture_replays_continue():
    """A CUDA graph captured around ks_step_n continues the simulation on each replay."""
    import torch
    w = wl.workload("plain_mix_8192", M=8)
    ens = ks.Ensemble(w)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ens.step(25, stream=torch.cuda.current_stream())
    # capture does not execute: step counter still 0
    torch.cuda.synchronize()
    assert int(ens.read_state(["step"])["step"][0]) == 0
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    got = ens.read_state()
    _, ref = _run_gpu(w, 75)
    for f in ref:
        if f != "trace":
            assert np.array_equal(got[f], ref[f]), f


def test_two_ensembles_double_buffered_on_two_streams():
    """The end-to-end pattern of the benchmark: two ensembles alternate on two
    streams, each step writing one ensemble's state from pinned host memory,
    launching it and reading the other's result while that launch runs.  Each
    ensemble then equals one ensemble run without interruption (and the oracle)."""
    import torch
    w = wl.workload("plain_mix_8192", M=12)
    chunk, rounds = 35, 2
    fields = ["order", "inventory", "cash", "last_tick", "history", "fundamental", "trades", "last_volume",
              "sum_price", "sum_volume", "trace_hash"]
    pair = (ks.Ensemble(w), ks.Ensemble(w))
    streams = (torch.cuda.Stream(), torch.cuda.Stream())
    views = [e.alloc_view(fields, pinned=True) for e in pair]
    ks.ks_read_state(pair[0].handle, views[0][0], streams[0])
    for f in fields:
        views[1][1][f].copy_(views[0][1][f])
    n = 2 * rounds
    for i in range(n):
        x = i % 2
        ks.ks_write_state(pair[x].handle, views[x][0], streams[x])
        ks.ks_step_n(pair[x].handle, chunk, streams[x])
        if i > 0:
            ks.ks_read_state(pair[1 - x].handle, views[1 - x][0], streams[1 - x])
    ks.ks_read_state(pair[(n - 1) % 2].handle, views[(n - 1) % 2][0], streams[(n - 1) % 2])
    for x in (0, 1):
        assert pair[x].sync(timeout_ms=600_000, stream=streams[x]) == ks.KS_OK
    ens, ref = _run_gpu(w, chunk * rounds)
    for x in (0, 1):
        got = {f: views[x][1][f].numpy() for f in fields}
        for f in fields:
            assert np.array_equal(got[f].view(ref[f].dtype).reshape(ref[f].shape), ref[f]), (x, f)
        assert int(pair[x].read_state(["step"])["step"][0]) == chunk * rounds
    oref = oracle_markets(w["params"], range(3), ens.L, ens.A, 0, chunk * rounds)
    for m, (mk, _, _) in oref.items():
        compare_market(ref, ens, m, mk)


@pytest.mark.parametrize("launch", [dict(threads=256, agents_per_thread=16),
                                    dict(threads=256, agents_per_thread=16, reg_cap=1)])
def test_policy_flag_written_into_rule_ensemble_is_ignored(launch):
    """An ensemble without a policy network ignores the MLP flag of written order
    words: its agents keep following their rule, and the flag stays in the word."""
    w = wl.workload("plain_mix_8192", M=6)
    ens, ref = _run_gpu(w, 40, launch=launch)
    e2 = ks.Ensemble(w)
    if launch:
        e2.set_launch(**launch)
    st = e2.read_state()
    st["order"] = st["order"] | np.uint32(1 << 23)
    e2.write_state(st)
    e2.step(40)
    assert e2.sync(timeout_ms=600_000) == ks.KS_OK
    got = e2.read_state()
    assert np.all(got["order"] & np.uint32(1 << 23))
    got["order"] = got["order"] & ~np.uint32(1 << 23)
    for f in ref:
        if f != "trace":
            assert np.array_equal(got[f], ref[f]), f


def test_full_size_plain_mix_sampled_markets():
    """8192 markets, L=1024, A=4096, 2000 steps in the bench's launch shape; sampled markets vs oracle."""
    w = wl.workload("plain_mix_8192")
    ens, gs = _run_gpu(w, w["S"])
    rng = np.random.default_rng(2)
    sample = sorted(set([0, w["M"] - 1] + list(rng.integers(0, w["M"], 2))))
    ref = oracle_markets(w["params"], sample, ens.L, ens.A, 0, w["S"])
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk)
    # ensemble-wide properties that hold at any size
    assert int(gs["inventory"].astype(np.int64).sum()) == 0
    assert int(gs["cash"].sum()) == 0
    assert np.all(gs["trades"] <= w["S"])


def test_error_word_clear_and_sync_deadline():
    import torch
    w = wl.workload("plain_mix_8192", M=4)
    ens = ks.Ensemble(w)
    ens.step(5)
    assert ens.sync(timeout_ms=60_000) == ks.KS_OK
    assert ks.ks_error_word(ens.handle) == 0
    torch.cuda.synchronize()


def test_plain_kernel_state_paths_on_uneven_offsets():
    """The plain kernel's 256-bit, 128-bit and scalar state paths: markets whose
    agent offsets fall on 32-byte, 16-byte and unaligned boundaries (offsets
    0, 4096, 8188, 9189, ... agents), every step against the oracle; then a
    zero-step launch (load, rebuild the book, store) leaves the state unchanged."""
    import torch
    As = np.array([4096, 4092, 1001, 4088, 8, 7, 4096, 2048], np.int32)
    Ls = np.full(len(As), 512, np.int32)
    w = wl.workload("plain_mix_8192", M=len(As))
    steps = 30
    ens, gs = _run_gpu(w, steps, trace_markets=len(As), launch=dict(threads=256, agents_per_thread=16), L=Ls, A=As)
    assert ens.batch_info()["batched"] == 0
    ref = oracle_markets(w["params"], range(len(As)), Ls, As, 0, steps)
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp, tv)
    before = ens.read_state()
    ks.ks_probe_state_io(ens.handle)
    torch.cuda.synchronize()
    after = ens.read_state()
    for f in before:
        assert np.array_equal(before[f], after[f]), f


@pytest.mark.parametrize("threads,ak,L,A", [(128, 8, 512, 700), (128, 16, 256, 1477),
                                            (256, 8, 512, 1100), (256, 16, 1024, 2955), (512, 8, 256, 3001),
                                            (512, 16, 512, 5909), (1024, 8, 256, 5000), (1024, 16, 256, 11818)])
def test_spreading_plain_variants(threads, ak, L, A):
    """A shape with room to spare runs the variant that spreads each market's
    agents over the CTA (ceil(A / threads) per thread): every market and step
    against the oracle, and the same state as the batched kernel, which
    spreads agents the same way."""
    M, steps = 3, 40
    w = wl.workload("plain_mix_8192", M=M, L=L, A=A)
    ens, gs = _run_gpu(w, steps, trace_markets=M, launch=dict(threads=threads, agents_per_thread=ak, reg_cap=1))
    assert ens.batch_info()["batched"] == 0
    ref = oracle_markets(w["params"], range(M), ens.L, ens.A, 0, steps)
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp, tv)


def test_spreading_plain_variant_on_uneven_markets():
    """Markets of 0 .. 4000 agents in one plain 256 x 16 launch (capacity 4096):
    each spreads its own agents; ragged ends and empty markets included."""
    As = np.array([4000, 0, 1, 255, 256, 257, 2049, 3999, 17, 4001], np.int32)
    Ls = np.array([1024, 64, 2, 128, 256, 512, 1024, 300, 40, 777], np.int32)
    w = wl.workload("plain_mix_8192", M=len(As))
    steps = 35
    ens, gs = _run_gpu(w, steps, trace_markets=len(As), launch=dict(threads=256, agents_per_thread=16, reg_cap=1),
                       L=Ls, A=As)
    assert ens.batch_info()["batched"] == 0
    ref = oracle_markets(w["params"], range(len(As)), Ls, As, 0, steps)
    for m, (mk, tp, tv) in ref.items():
        compare_market(gs, ens, m, mk, tp, tv)
