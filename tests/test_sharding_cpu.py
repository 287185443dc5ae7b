"""The multi-GPU launch path on CPU: two gloo ranks shard the global market
index space with no data-path collective and max-reduce their timings."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    from paper_2606_21784_gb300 import sharding, workloads
    r, w = sharding.init("gloo")
    wl = sharding.shard(workloads.workload("plain_mix_8192"), r, w)
    sharding.barrier()
    t = sharding.max_over_ranks(1.5 + rank)
    total = sharding.sum_over_ranks(float(wl["M"]))
    q.put((rank, wl["market_base"], wl["M"], t, total))
    sharding.finalize()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_shard_and_reduce(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    M = out[0][2]
    bases = [o[1] for o in out]
    assert bases == [r * M for r in range(world)]          # disjoint global market ranges
    assert all(o[3] == 1.5 + (world - 1) for o in out)      # time = max over ranks
    assert all(o[4] == world * M for o in out)              # weak scaling: work grows with ranks


def _oracle_rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle as o
    from paper_2606_21784_gb300 import sharding, workloads
    r, w = sharding.init("gloo")
    part = sharding.shard(workloads.workload("plain_mix_8192", M=3, L=64, A=96), r, w)
    mine = []
    for i in range(part["M"]):
        g = part["market_base"] + i
        mk, tp, tv = o.simulate(part["params"], g, 64, 96, 25)
        mine.append((g, mk.scalars()["hash"], int(mk.inv.sum()), tp.tolist()))
    got = [None] * w
    dist.all_gather_object(got, mine)
    q.put((rank, got))
    sharding.finalize()


def test_two_gloo_ranks_reproduce_a_one_rank_run():
    """Each of two gloo ranks runs the oracle on its shard of the global market
    range (no data-path collective); the per-market results gathered at the
    end equal a single run over all 2M markets: the same trace hashes, traces
    and conserved inventories for every global market index."""
    import oracle as o
    from paper_2606_21784_gb300 import workloads
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered = sorted(x for per_rank in out[0][1] for x in per_rank)
    assert out[0][1] == out[1][1]
    w = workloads.workload("plain_mix_8192", M=3 * world, L=64, A=96)
    single = []
    for g in range(w["M"]):
        mk, tp, tv = o.simulate(w["params"], g, 64, 96, 25)
        single.append((g, mk.scalars()["hash"], int(mk.inv.sum()), tp.tolist()))
    assert [x[0] for x in gathered] == list(range(w["M"]))  # disjoint shards cover the range
    assert gathered == single
    assert all(x[2] == 0 for x in single)
    assert len({x[1] for x in single}) == w["M"]  # markets differ: the global index keys the draws


def test_single_process_defaults():
    from paper_2606_21784_gb300 import sharding, workloads
    r, w, lr = sharding.rank_env()
    assert (r, w) == (0, 1) or "RANK" in os.environ
    wl = sharding.shard(workloads.workload("plain_zi_64"), 0, 1)
    assert wl["market_base"] == 0
    assert sharding.max_over_ranks(3.0) == 3.0


def test_reference_arm_under_torchrun_prints_one_line():
    """The reference arm as the scaling run launches it: two ranks through
    torch.distributed.run; rank 0 alone times the oracle and prints one JSON
    line, the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1", "--sim-steps", "5"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
