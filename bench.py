#!/usr/bin/env python
"""Benchmark of the persistent call-auction kernel: agent events per second.

One bench step = one ks_step_n over the whole ensemble for the workload's S
steps (default: 8192 markets, L=1024, A=4096, S=2000; state 512 MiB resident
in HBM, larger than L2).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank simulates its own range of global market indices
(weak scaling, no data-path collective); the time is the max over ranks.
``--impl reference`` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PHILOX_MULW_PER_EVENT = 20  # Philox4x32-10: 10 rounds x 2 32x32->64 products per agent-event
SM_COUNT_NOMINAL = 152
SM_MAX_MHZ_NOMINAL = 2070.0
PROFILE = os.path.join(ROOT, "profiles", "plain_kernel_plain_mix_8192.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain_mix_8192")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probes", action="store_true")
    ap.add_argument("--sim-steps", type=int, default=0, help="override S (profiling small cases)")
    ap.add_argument("--markets", type=int, default=0, help="override M (profiling small cases)")
    ap.add_argument("--launch", default="",
                    help="threads,agents_per_thread,reg_cap (paper workloads: threads,agents_per_thread,min_ctas); "
                         "skips the autotuner")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched / learned comparison runs")
    ap.add_argument("--engine", default="persistent", choices=["persistent", "naive"],
                    help="paper-agent workloads: the persistent kernel or the naive one-thread-per-market engine")
    return ap.parse_args()


PLAIN_SOURCES = ("ks_device.cuh", "ks_internal.h", "ks_market.cuh", "ks_plain.cuh")


def strip_comments(src: str) -> str:
    """C/C++ source without comments and whitespace (string and character literals kept)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            if not c.isspace():
                out.append(c)
            i += 1
    return "".join(out)


def kernel_source_hash(d: str | None = None) -> str:
    """Hash of the plain kernel's code (comments and whitespace removed); ncu counters are
    only valid for the kernel they were taken on."""
    h = hashlib.sha256()
    d = d or os.path.join(ROOT, "paper_2606_21784_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        if fn in PLAIN_SOURCES or fn.startswith("ks_plain_nt") or fn == "ks_plain_carried.cu":
            h.update(fn.encode())
            h.update(strip_comments(open(os.path.join(d, fn), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch recorded in the committed ncu summary, if it matches the current sources."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # nvidia-smi's start-up (NVML init) can stall CUDA calls of this
        # process for seconds: wait for its first sample so that the stall
        # falls before the timed region, not inside it
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < 20.0:
            if os.path.getsize(self.path) > 0 or self.proc.poll() is not None:
                break
            time.sleep(0.05)
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle (the reported CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_market(args):
    params, m, L, A, S = args
    import oracle as o
    mk = o.init_market(params, m, L, A)
    t = time.perf_counter()
    o.run_market(params, mk, 0, S, want_trace=False)
    return time.perf_counter() - t


def _oracle_warm(_):
    import oracle as o
    o.philox4x32_10([0, 0, 0, 0], [0, 0])
    return 0


def oracle_sample(w: dict, markets_per_core: int = 2):
    """Runs the oracle on `cores x markets_per_core` markets of workload w over
    all S steps, one market per task on a spawn pool of all host cores."""
    import multiprocessing as mp

    from paper_2606_21784_gb300 import workloads
    import oracle  # noqa: F401  (builds the C oracle before the pool starts)
    oracle.build()
    cores = os.cpu_count() or 1
    L, A = workloads.sizes(w)
    n = min(len(L), cores * markets_per_core)
    step = max(1, len(L) // n)
    idx = [i * step for i in range(n)]
    tasks = [(w["params"], int(m) + int(w.get("market_base", 0)), int(L[m]), int(A[m]), int(w["S"])) for m in idx]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_warm, range(cores))  # worker start-up and library load stay outside the timing
        t = time.perf_counter()
        task_s = pool.map(_oracle_market, tasks, chunksize=1)
        dt = time.perf_counter() - t
    events = float(sum(int(A[m]) for m in idx)) * w["S"]
    # one core's rate: the events over the summed per-market times (each task
    # ran on one core, with the other cores busy)
    single = events / max(sum(task_s), 1e-9)
    return events / dt, cores, f"{n} markets x {w['S']} steps ({int(events):d} agent-events), one market per task", \
        events, single


def _oracle_market_mlp(args):
    params, m, L, A, S, mlp_w = args
    import oracle as o
    mk = o.init_market(params, m, L, A)
    t = time.perf_counter()
    o.run_market(params, mk, 0, S, want_trace=False, mlp_w=mlp_w)
    return time.perf_counter() - t


def oracle_bucket_sample(w: dict, L, A, S: int, mlp_w=None, per_bucket: int = 1):
    """The oracle's rate on a sample of workload w that covers every power-of-two
    (L, A) class: `per_bucket` markets of each class (the first ones), S steps
    each, one market per task on a spawn pool of all host cores.  Policy agents
    decide with the fp64 network `mlp_w`."""
    import multiprocessing as mp

    import numpy as np

    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    classes = {}
    for m, (l, a) in enumerate(zip(L, A)):
        key = (1 << max(0, int(l) - 1).bit_length(), 1 << max(0, int(a) - 1).bit_length())
        if len(classes.setdefault(key, [])) < per_bucket:
            classes[key].append(m)
    idx = sorted(m for ms in classes.values() for m in ms)
    base = int(w.get("market_base", 0))
    tasks = [(w["params"], m + base, int(L[m]), int(A[m]), S, mlp_w) for m in idx]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_warm, range(cores))
        t = time.perf_counter()
        task_s = pool.map(_oracle_market_mlp, tasks, chunksize=1)
        dt = time.perf_counter() - t
    events = float(np.sum([int(A[m]) for m in idx])) * S
    return {"value": events / dt, "unit": "events/s", "cores": cores, "kind": "oracle",
            "single_core_value": events / max(sum(task_s), 1e-9),
            "sample": f"{len(idx)} markets ({len(classes)} (L, A) classes x up to {per_bucket}) x {S} steps "
                      f"({int(events):d} agent-events), one market per task"}


def run_reference(args):
    from paper_2606_21784_gb300 import sharding, workloads
    rank, world, _ = sharding.rank_env()
    if rank != 0:
        return 0
    w = workloads.workload(args.workload)
    if args.sim_steps:
        w["S"] = args.sim_steps
    per_core = 1
    vals, singles = [], []
    for i in range(args.warmup + args.steps):
        v, cores, sample, events_per_step, single = oracle_sample(w, per_core)
        if i >= args.warmup:
            vals.append(v)
            singles.append(single)
    value = statistics.median(vals)
    out = {
        "impl": "reference", "metric": "agent_events_per_s", "value": value, "unit": "events/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": events_per_step / value * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "M": w["M"], "S": w["S"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "single_core_value": statistics.median(singles)},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def time_probe(ks, kind, blocks, iters, sink, stream, reps=3):
    import torch
    ks.ks_probe(kind, blocks, max(1, iters // 10), sink.data_ptr(), stream)
    best = None
    ops = 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ops = ks.ks_probe(kind, blocks, iters, sink.data_ptr(), stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return ops / (best / 1e3)


def _time_ensemble(ens, steps, stream):
    import torch
    ens.step(max(1, steps // 10), stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.step(steps, stream)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def _graph_of(ens, S):
    """One S-step ks_step_n captured in a CUDA graph (on a capture stream of
    its own; the graph is replayed on the timing stream)."""
    import torch
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=torch.cuda.Stream()):
        ens.step(S, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return g


def _time_graph(g, stream, reps=1):
    import torch
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            g.replay()
            e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best / 1e3


def compare_forms(ks, workloads, stream, plain_rate, cpu=True):
    """Throughput of the other forms of the method on the same GPU, each on
    the configuration it is stated for, beside the plain persistent kernel:
    the batched uneven ensemble (20000 markets, S=2000, one launch, default
    and tuned plan), and the learned-agent forms with the network trained by
    behaviour cloning on 20M pairs (4096 all-policy markets at S=2000; 32768
    uneven markets with 25% policy agents at S=10000 as one CUDA-graph-captured
    launch beside the same instances with rule agents only).  With `cpu`,
    each form also gets the oracle's rate on a sample of one market per
    (L, A) class."""
    import numpy as np
    out = {"plain_mix_8192": {"events_per_s": plain_rate}}
    w = workloads.workload("batched_20000")
    L, A = workloads.sizes(w)
    S = int(w["S"])
    ens = ks.Ensemble(w, L=L, A=A)
    ev = float(A.astype(np.int64).sum()) * S
    info = ens.batch_info()
    out["batched_20000"] = {"events_per_s": ev / _time_ensemble(ens, S, stream), "steps": S,
                            "agent_events_per_launch": ev, "plan": "default", "items": info["n_items"],
                            "buckets": info["n_buckets"], "cta_threads": info["cta_threads"],
                            "vs_plain": None}
    out["batched_20000"]["vs_plain"] = out["batched_20000"]["events_per_s"] / plain_rate
    try:
        from paper_2606_21784_gb300 import autotune
        plan = autotune.tune_batched(w, L, A)
        if plan["buckets"] is not None:
            ens.set_batch_plan(plan["cta_threads"], plan["buckets"])
        out["batched_20000_tuned"] = {"events_per_s": ev / _time_ensemble(ens, S, stream), "steps": S,
                                      "cta_threads": plan["cta_threads"],
                                      "kept_default": plan["buckets"] is None}
    except Exception as e:  # the tuned plan is optional; the default plan was measured above
        out["batched_20000_tuned"] = {"error": str(e)[:200]}
    ens.close()
    if cpu:
        out["batched_20000"]["cpu_baseline"] = oracle_bucket_sample(w, L, A, S)
    out.update(learned_forms(ks, workloads, stream, cpu=cpu))
    out["cda_8192"] = cda_form(ks, workloads, stream, cpu=cpu)
    out["paper_table_iii"] = paper_forms(ks, workloads, stream)
    out["paper_stylized_facts"] = stylized_facts()
    return out


def _oracle_cda_market(args):
    params, m, L, A, S = args
    import oracle as o
    mk = o.cda_init(params, m, L, A)
    t = time.perf_counter()
    o.cda_run(params, mk, 0, S)
    return time.perf_counter() - t


def cda_form(ks, workloads, stream, cpu=True, reps=2):
    """The continuous double auction over the configuration's agents (8192
    markets x 1024 agents x 1024 ticks, S=500, one launch), and the oracle on
    one market per host core."""
    import multiprocessing as mp

    import torch
    w = workloads.workload("cda_8192")
    S = int(w["S"])
    ens = ks.CdaEnsemble(w)
    ens.step(20, stream)
    torch.cuda.synchronize()
    best = _time_best(lambda: ens.step(S, stream), stream, reps)
    if ens.sync(timeout_ms=600_000) != ks.KS_OK:
        raise RuntimeError("CDA ensemble reported a device error")
    st = ens.read_state(["fills"])
    ev = float(w["M"]) * w["A"] * S
    out = {"events_per_s": ev / (best / 1e3), "ms_per_run": best, "steps": S,
           "fills_per_market_step": float(st["fills"].mean()) / (S * reps + 20),
           "roofline": cda_roofline(ev, best)}
    ens.close()
    if cpu:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        tasks = [(w["params"], m, int(w["L"]), int(w["A"]), S) for m in range(cores)]
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(_oracle_warm, range(cores))
            t = time.perf_counter()
            task_s = pool.map(_oracle_cda_market, tasks, chunksize=1)
            dt = time.perf_counter() - t
        cev = float(cores) * w["A"] * S
        out["cpu_baseline"] = {"value": cev / dt, "unit": "events/s", "cores": cores, "kind": "oracle",
                               "single_core_value": cev / max(sum(task_s), 1e-9),
                               "sample": f"{cores} markets x {S} steps, one market per task"}
    return out


def stylized_facts():
    """The paper's market-composition sweep (alpha_mom 0..0.70, alpha_maker
    0.15, 64 markets x 1000 steps, A=256, L=128) with the paper's own agent
    model, on a sliding window and on a fixed grid: volatility, excess
    kurtosis, volume per step and lag-1 autocorrelations per configuration,
    and the sweep's device time (the paper quotes under 0.25 s for its
    sweep)."""
    from paper_2606_21784_gb300 import dynamics

    def rows(r):
        return {f"{a:.2f}": {"volatility": round(f["volatility"], 3), "price_std": round(f["price_std"], 2),
                             "excess_kurtosis": round(f["excess_kurtosis"], 2),
                             "volume_per_step": round(f["volume_per_step"], 1), "acf_r_lag1": round(f["acf_r"][0], 3),
                             "acf_abs_r_lag1": round(f["acf_abs_r"][0], 3)} for a, f in r["facts"].items()}
    r = dynamics.sweep()
    fixed = dynamics.sweep(window=False)
    return {"by_alpha_mom": rows(r), "by_alpha_mom_fixed_grid": rows(fixed), "device_seconds": r["device_seconds"],
            "agent_events": r["agent_events"],
            "paper_values": {k: {str(a): v for a, v in d.items()} for k, d in dynamics.PAPER_FACTS.items()}}


# the shapes of the paper's throughput table (markets sweep at A=256, agents
# sweep at 8192 markets; L=128, S=500)
PAPER_SHAPES = ((64, 256), (256, 256), (1024, 256), (4096, 256), (16384, 256), (8192, 16), (8192, 64), (8192, 256),
                (8192, 1024))
# the paper's peak throughput (RTX 5090, its own agents, Table III): context for the paper workloads' line only
PAPER_PEAK = {(8192, 1024): 5.47e10}


def _time_best(run, stream, reps):
    import torch
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def paper_forms(ks, workloads, stream, reps: int = 3):
    """The paper's own agent model (tick-aggregated book, NOISE / MOMENTUM /
    MAKER agents, SplitMix64 draws) on the shapes of the paper's throughput
    table, each with its tuned launch, and the naive engine (one thread per
    market, book in global memory, one launch per step) on the same shapes:
    the paper's ablation of its two design choices, on this GPU."""
    import torch

    from paper_2606_21784_gb300 import autotune
    out = {}
    for (M, A) in PAPER_SHAPES:
        w = workloads.workload("paper_8192_256", M=M, A=A)
        ens = ks.PaperEnsemble(w)
        launch = autotune.apply(ens, w)
        S = int(w["S"])
        ens.step(50, stream)
        torch.cuda.synchronize()
        best = _time_best(lambda: ens.step(S, stream), stream, reps)
        ens.step_naive(5, stream)
        torch.cuda.synchronize()
        naive = _time_best(lambda: ens.step_naive(S, stream), stream, reps)
        if ens.sync(timeout_ms=600_000) != ks.KS_OK:
            raise RuntimeError("paper ensemble reported a device error")
        ev = float(M) * A * S
        rate, nrate = ev / (best / 1e3), ev / (naive / 1e3)
        out[f"M{M}_A{A}"] = {"events_per_s": rate, "ms_per_run": best,
                             "launch": {k: launch[k] for k in ("threads", "agents_per_thread", "min_ctas")},
                             "naive_events_per_s": nrate, "speedup_over_naive": rate / nrate}
        if (M, A) == (4096, 256):
            out["step_latency_us_4096x256"] = {"persistent": 1e3 * best / S, "naive": 1e3 * naive / S}
        ens.close()
    return out


def trained_policy(pairs: int = 20_000_000, epochs: int = 3):
    """The policy trained by behaviour cloning on `pairs` (state, action) pairs
    of the rule-based 8192-market run with seed 7, with the library's
    tensor-core training kernels; returns (blob, report)."""
    import time

    import torch

    from paper_2606_21784_gb300 import bc
    t0 = time.time()
    rec, wd = bc.generate(pairs)
    torch.cuda.synchronize()
    t1 = time.time()
    params, hist, val = bc.train(rec, wd["A"], epochs=epochs)
    torch.cuda.synchronize()
    t2 = time.time()
    blob = bc.export(params)
    n_train = int(rec.shape[0]) - int(val.shape[0])
    rep = {"pairs": int(rec.shape[0]), "epochs": epochs, "generate_s": t1 - t0, "train_s": t2 - t1,
           "train_pairs_per_s": n_train * epochs / max(t2 - t1, 1e-9),
           "held_out_loss": {"trained": hist["val_loss"][-1],
                             "input_independent": bc.evaluate(bc.marginal_params(rec), val, wd["A"]),
                             "untrained": hist["val_loss"][0]},
           "val_loss_by_epoch": hist["val_loss"]}
    del rec
    torch.cuda.synchronize()
    return blob, params, rep


# algorithmic FLOP of one policy decision: 2 * (32*64 + 64*64 + 64*37)
POLICY_FLOP = 2 * (32 * 64 + 64 * 64 + 64 * 37)


def learned_forms(ks, workloads, stream, cpu=True):
    """The learned-agent forms on their stated configurations: a policy trained
    by behaviour cloning on 20M (state, action) pairs of the rule-based seed-7
    run, then (a) the 4096-market all-policy ensemble at S=2000 and (b) the
    32768-market uneven ensemble with 25% policy agents at S=10000, one
    CUDA-graph-captured launch, beside the same instances with rule agents
    only (also one captured launch).  The tensor-pipe fraction counts the
    network's algorithmic FLOP per decision (17,024) against the measured
    sustained BF16 peak."""
    import numpy as np
    import torch

    from paper_2606_21784_gb300 import autotune
    out = {}
    blob, params, rep = trained_policy()
    out["bc"] = rep
    peaks = measured_peaks()
    tc_peak = peaks.get("bf16_tflops_sustained") or 1700.0
    w = workloads.workload("learned_4096")
    S = int(w["S"])
    ens = ks.Ensemble(w, mlp_params=blob)
    autotune.apply(ens, w)
    cap = ens.set_capture(count_policy=True)
    ev = float(w["M"]) * w["A"] * S
    ens.step(20, stream)
    torch.cuda.synchronize()
    cap["policy_count"].zero_()
    dt = _time_ensemble(ens, S, stream)
    dec = float(cap["policy_count"].item()) * S / (S + S // 10)  # warm-up steps excluded
    tflops = dec * POLICY_FLOP / dt / 1e12
    out["learned_4096"] = {"events_per_s": ev / dt, "steps": S, "agent_events_per_launch": ev,
                           "policy_decisions_per_s": dec / dt, "launch": ens.get_launch(),
                           "tensor_roofline": {"bound": "tensor", "achieved": tflops, "peak": tc_peak,
                                               "unit": "TFLOP/s", "frac": tflops / tc_peak,
                                               "algorithmic": f"{POLICY_FLOP} FLOP per policy decision",
                                               "peak_source": "measured sustained BF16 (MEASURED_PEAKS.json)"}}
    ens.close()
    w = workloads.workload("mixed_32768")
    L, A = workloads.sizes(w)
    S = int(w["S"])
    ev = float(A.astype(np.int64).sum()) * S
    for pct in (25, 0):
        ww = workloads.workload("mixed_32768", mlp_pct=pct)
        e2 = ks.Ensemble(ww, L=L, A=A, mlp_params=blob if pct else None)
        if pct:
            cap = e2.set_capture(count_policy=True)
        e2.step(50, stream)
        torch.cuda.synchronize()
        g = _graph_of(e2, S)
        if pct:
            cap["policy_count"].zero_()
        dt = _time_graph(g, stream)
        if e2.sync(timeout_ms=600_000) != ks.KS_OK:
            raise RuntimeError("mixed ensemble reported a device error")
        r = {"events_per_s": ev / dt, "steps": S, "agent_events_per_launch": ev, "graph_captured": True,
             "cta_threads": e2.batch_info()["cta_threads"]}
        if pct:
            dec = float(cap["policy_count"].item())
            tflops = dec * POLICY_FLOP / dt / 1e12
            r["policy_decisions_per_s"] = dec / dt
            r["tensor_roofline"] = {"bound": "tensor", "achieved": tflops, "peak": tc_peak, "unit": "TFLOP/s",
                                    "frac": tflops / tc_peak}
        out[f"mixed_32768_policy{pct}"] = r
        del g
        e2.close()
    out["mixed_32768_policy25"]["vs_rule_only"] = (out["mixed_32768_policy25"]["events_per_s"]
                                                   / out["mixed_32768_policy0"]["events_per_s"])
    if cpu:
        w64 = policy_fp64(ks, params)
        wl4 = workloads.workload("learned_4096")
        out["learned_4096"]["cpu_baseline"] = oracle_bucket_sample(
            wl4, *workloads.sizes(wl4), 100, mlp_w=w64, per_bucket=16)
        out["mixed_32768_policy25"]["cpu_baseline"] = oracle_bucket_sample(
            workloads.workload("mixed_32768"), L, A, 200, mlp_w=w64)
    return out


def policy_fp64(ks, params):
    """The fp64 parameter vector the oracle decides with: the trained FP32
    parameters with the weights rounded to BF16, as the kernels use them."""
    import oracle as o
    parts = o.mlp_unpack(params.double().cpu().numpy())
    return o.mlp_pack(*ks.mlp_params_as_used(*parts))


def e2e_double_buffered(ks, w, L_, A_, blob, ens, configure, fields, bufs, S, steps, sharding, dev):
    """End to end through the C ABI with two ensembles of the same workload on
    two streams.  Step i writes ensemble i % 2's state from pinned host memory,
    queues its S-step launch, then reads the other ensemble's result of step
    i - 1, so that one ensemble's copies run while the other's kernel does;
    every step still moves its whole state in and out.  Both ensembles start
    from the host state in ``bufs``.  Returns (seconds, steps), the time being
    the max over ranks."""
    import torch

    ens2 = ks.Ensemble(w, L=L_, A=A_, mlp_params=blob)
    configure(ens2)  # the same launch shape or batch plan as `ens`
    pair = (ens, ens2)
    streams = (torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev))
    views = []
    for e in pair:
        v, b = e.alloc_view(fields, pinned=True)
        for f in fields:
            b[f].copy_(bufs[f])
        views.append(v)
    # one untimed round trip per ensemble: first use of its streams and buffers
    for x in (0, 1):
        ks.ks_write_state(pair[x].handle, views[x], streams[x])
        ks.ks_step_n(pair[x].handle, S, streams[x])
        ks.ks_read_state(pair[x].handle, views[x], streams[x])
    torch.cuda.synchronize()
    sharding.barrier()
    t0 = time.perf_counter()
    for i in range(steps):
        x = i % 2
        ks.ks_write_state(pair[x].handle, views[x], streams[x])       # host -> device (syncs its stream)
        ks.ks_step_n(pair[x].handle, S, streams[x])
        if i > 0:
            ks.ks_read_state(pair[1 - x].handle, views[1 - x], streams[1 - x])  # device -> host (syncs)
    y = (steps - 1) % 2
    ks.ks_read_state(pair[y].handle, views[y], streams[y])
    secs = sharding.max_over_ranks(time.perf_counter() - t0, dev)
    for x in (0, 1):
        if pair[x].sync(timeout_ms=600_000, stream=streams[x]) != ks.KS_OK:
            raise RuntimeError("double-buffered end-to-end run reported an error")
    ens2.close()
    return secs, steps


def run_ours(args):
    import numpy as np
    import torch

    from paper_2606_21784_gb300 import kineticsim as ks
    from paper_2606_21784_gb300 import sharding, workloads

    rank, world, local_rank = sharding.rank_env()
    torch.cuda.set_device(local_rank)
    sharding.init("nccl")
    dev = torch.device("cuda", local_rank)

    w = workloads.workload(args.workload)
    if args.sim_steps:
        w["S"] = args.sim_steps
    if args.markets:
        w["M"] = args.markets
    w = sharding.shard(w, rank, world)
    if w.get("model") == "paper":
        return run_paper(args, w, rank, world, dev)
    if w.get("model") == "cda":
        return run_cda(args, w, rank, world, dev)
    S = int(w["S"])
    blob = trained_policy(2_000_000, 1)[0] if int(w["params"].get("mlp_pct", 0)) > 0 else None
    L_, A_ = workloads.sizes(w)
    ens = ks.Ensemble(w, L=L_, A=A_, mlp_params=blob)
    def configure(e):
        if args.launch:
            nt, ak, rc = (int(x) for x in args.launch.split(","))
            e.set_launch(nt, ak, reg_cap=rc)
        else:
            from paper_2606_21784_gb300 import autotune
            autotune.apply(e, w)

    configure(ens)
    launch = ens.get_launch()
    L, A = ens.L, ens.A
    events_per_step = float(A.astype(np.int64).sum()) * S
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        ens.step(S, stream)
    torch.cuda.synchronize()
    sharding.barrier()

    sampler = ClockSampler(local_rank)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for e0, e1 in ev:
        e0.record(stream)
        ens.step(S, stream)
        e1.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    sharding.barrier()
    clocks = sampler.stop()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms_max = sharding.max_over_ranks(total_ms, dev)
    value = world * events_per_step * args.steps / (total_ms_max / 1e3)
    st = ens.sync(timeout_ms=600_000)
    if st != ks.KS_OK:
        raise RuntimeError(f"ensemble reported status {st}")

    # end to end through the C ABI with pinned host buffers
    fields = ["order", "inventory", "cash", "last_tick", "history", "fundamental", "trades", "last_volume",
              "sum_price", "sum_volume", "trace_hash"]
    view, bufs = ens.alloc_view(fields, pinned=True)
    ks.ks_read_state(ens.handle, view, stream)
    state_bytes = sum(t.numel() * t.element_size() for t in bufs.values())
    # one untimed round trip first: the clock sampler's shutdown and the first
    # use of the pinned buffers fall before the timed region
    ks.ks_write_state(ens.handle, view, stream)
    ks.ks_step_n(ens.handle, S, stream)
    ks.ks_read_state(ens.handle, view, stream)
    torch.cuda.synchronize()
    sharding.barrier()
    t0 = time.perf_counter()
    phases = []
    for _ in range(args.e2e_steps):
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        a = time.perf_counter()
        ks.ks_write_state(ens.handle, view, stream)   # host -> device: the step's inputs (syncs)
        b = time.perf_counter()
        k0.record(stream)
        ks.ks_step_n(ens.handle, S, stream)
        k1.record(stream)
        ks.ks_read_state(ens.handle, view, stream)    # device -> host: the step's result (syncs)
        phases.append((b - a, time.perf_counter() - b, k0.elapsed_time(k1) / 1e3))
    e2e_s = time.perf_counter() - t0
    e2e_s = sharding.max_over_ranks(e2e_s, dev)
    seq_value = world * events_per_step * args.e2e_steps / e2e_s
    pipe_s, pipe_steps = e2e_double_buffered(ks, w, L_, A_, blob, ens, configure, fields, bufs, S,
                                             max(4, args.e2e_steps), sharding, dev)
    e2e_value = world * events_per_step * pipe_steps / pipe_s

    mean_launch_s = statistics.mean(launch_ms) / 1e3
    out = None
    if rank == 0:
        probes = {}
        if not args.no_probes:
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            sink = torch.empty(sms * 8 * 256 * 8, dtype=torch.uint8, device=dev)
            probes["smem_red_ops_per_s"] = time_probe(ks, ks.KS_PROBE_SMEM_RED, sms * 8, 20000, sink, stream)
            probes["mul_wide_per_s"] = time_probe(ks, ks.KS_PROBE_MUL_WIDE, sms * 8, 100000, sink, stream)
            probes["mul_hilo_per_s"] = time_probe(ks, ks.KS_PROBE_MUL_HILO, sms * 8, 100000, sink, stream)
            probes["philox_blocks_per_s"] = time_probe(ks, ks.KS_PROBE_PHILOX, sms * 8, 20000, sink, stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            ks.ks_probe_state_io(ens.handle, stream)
            e0.record(stream)
            io_bytes = ks.ks_probe_state_io(ens.handle, stream)
            e1.record(stream)
            e1.synchronize()
            probes["state_io_gbs"] = io_bytes / (e0.elapsed_time(e1) / 1e3) / 1e9
            probes["sms"] = sms
        peaks = measured_peaks()
        # ALU roofline: Philox needs 20 32 x 32 -> 64 products per agent-event;
        # the per-SM rate R is the faster probe's (one mad.wide.u32, or a
        # mul.hi and a mul.lo, per product), rounded to a power of two at the
        # sampled clock; the peak is 152 SMs x R x 2070 MHz.
        sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1455.0
        R = None
        rates = [probes[k] for k in ("mul_wide_per_s", "mul_hilo_per_s") if k in probes]
        if rates:
            r = max(rates) / (probes["sms"] * sm_mhz * 1e6)
            R = 2 ** round(np.log2(r))
        achieved = PHILOX_MULW_PER_EVENT * events_per_step / mean_launch_s / 1e12
        roofline = None
        if R:
            peak = SM_COUNT_NOMINAL * R * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
            tr = profiled_traffic()
            roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tproducts/s",
                        "frac": achieved / peak, "traffic": tr,
                        "peak_source": f"derived: {SM_COUNT_NOMINAL} SMs x {R} products/clk/SM "
                                       f"(per-SM rate of the faster product probe, mul.wide or mul.hi + mul.lo) "
                                       f"x {SM_MAX_MHZ_NOMINAL:.0f} MHz",
                        "algorithmic": f"{PHILOX_MULW_PER_EVENT} 32x32->64 products per agent-event x "
                                       f"{events_per_step:.4g} agent-events per launch",
                        "kernel": "plain_kernel", "launch_ms": statistics.mean(launch_ms)}
        rooflines = {}
        ev_rate_launch = events_per_step / mean_launch_s
        if "smem_red_ops_per_s" in probes:
            rooflines["smem_atomic"] = {"achieved_events_per_s": ev_rate_launch,
                                        "peak_lane_atomics_per_s": probes["smem_red_ops_per_s"],
                                        "frac": ev_rate_launch / probes["smem_red_ops_per_s"],
                                        "note": "1 aggregated order per agent-event against measured "
                                                "conflict-free red.shared.add.u32 throughput"}
            rooflines["philox_rate"] = {"achieved_events_per_s": ev_rate_launch,
                                        "peak_blocks_per_s": probes["philox_blocks_per_s"],
                                        "frac": ev_rate_launch / probes["philox_blocks_per_s"]}
            hbm = peaks.get("hbm_gbs", 6800.0)
            rooflines["state_io_hbm"] = {"achieved": probes["state_io_gbs"], "peak": hbm, "unit": "GB/s",
                                         "frac": probes["state_io_gbs"] / hbm,
                                         "note": "zero-step launch: load + store of 32 B per agent"}
        forms = {}
        if not args.no_forms and world == 1:
            forms = compare_forms(ks, workloads, stream, ev_rate_launch)
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            v, cores, sample, _, single = oracle_sample(w, 2)
            cpu = {"value": v, "unit": "events/s", "cores": cores, "kind": "oracle", "sample": sample,
                   "single_core_value": single}
        out = {
            "metric": "agent_events_per_s", "value": value, "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "M": int(w["M"]), "L": int(L.max()), "A": int(A.max()),
                       "S": S, "agent_events_per_step": events_per_step,
                       "l2": f"inputs larger than L2 (resident state {state_bytes / 2**20:.0f} MiB)",
                       "launch": launch, "parallelism": f"markets sharded over {world} GPU(s)"},
            "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes,
                    "mode": f"double-buffered: two ensembles on two streams, {pipe_steps} steps; each step "
                            f"writes one ensemble's state, queues its launch and reads the other's result "
                            f"while that launch runs.  Consecutive launches of the two ensembles also overlap "
                            f"at their tails (the next launch's CTAs start on SMs the last markets of the "
                            f"previous one leave idle), so the rate can exceed back-to-back launches on one "
                            f"stream",
                    "sequential": {
                        "value": seq_value, "steps": args.e2e_steps,
                        "mode": "one ensemble: write, step, read, each step after the previous one",
                        "breakdown_ms": {
                            "write_state": round(1e3 * statistics.median(p[0] for p in phases), 2),
                            "step_and_read_state": round(1e3 * statistics.median(p[1] for p in phases), 2),
                            "kernel_in_round_trip": round(1e3 * statistics.median(p[2] for p in phases), 2),
                            "device_launch": round(1e3 * mean_launch_s, 2)}}},
            "gpu_launches": 2 * args.steps,
            "roofline": roofline,
            "rooflines": rooflines,
            "probes": probes,
            "cpu_baseline": cpu,
            "forms": forms,
            "clocks": clocks,
            "paper_context": {"value": 5.47e10, "hardware": "RTX 5090 (sm_120), L=128, S=500, M=8192, A=1024"},
        }
        print(json.dumps(out), flush=True)
    ens.close()
    sharding.finalize()
    return 0


def run_paper(args, w, rank, world, dev):
    """The paper's own agent model as the main workload (``--workload
    paper_*``): same timing rules; the state is read back to the host in the
    end-to-end leg (the model has no per-agent state to upload)."""
    import torch

    from paper_2606_21784_gb300 import autotune
    from paper_2606_21784_gb300 import kineticsim as ks
    from paper_2606_21784_gb300 import sharding
    ens = ks.PaperEnsemble(w)
    if args.launch:
        nt, ak, mc = (int(x) for x in args.launch.split(","))
        ens.set_launch(nt, ak, mc)
    else:
        autotune.apply(ens, w)
    S = int(w["S"])
    events_per_step = float(w["M"]) * w["A"] * S
    naive = args.engine == "naive"
    run = ens.step_naive if naive else ens.step  # the naive engine: one launch per simulated step
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        run(S, stream)
    torch.cuda.synchronize()
    sharding.barrier()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0e = torch.cuda.Event(enable_timing=True)
    t1e = torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    for e0, e1 in ev:
        e0.record(stream)
        run(S, stream)
        e1.record(stream)
    t1e.record(stream)
    torch.cuda.synchronize()
    sharding.barrier()
    clocks = sampler.stop()
    total_ms = sharding.max_over_ranks(t0e.elapsed_time(t1e), dev)
    value = world * events_per_step * args.steps / (total_ms / 1e3)
    if ens.sync(timeout_ms=600_000) != ks.KS_OK:
        raise RuntimeError("paper ensemble reported a device error")
    run(S, stream)  # one untimed round trip first, as in the main workload
    ens.read_state(["bid", "ask", "last_tick", "trades", "sum_volume"], stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nbytes = 0
    for _ in range(args.e2e_steps):
        run(S, stream)
        st = ens.read_state(["bid", "ask", "last_tick", "trades", "sum_volume"], stream)
        nbytes = sum(a.nbytes for a in st.values())
    e2e_s = sharding.max_over_ranks(time.perf_counter() - t0, dev)
    roofline = None
    if rank == 0 and not naive and not args.no_probes:
        # ALU roofline: two SplitMix64 mixes per agent-event against the mix
        # rate of a pure loop of the kernel's own mix routine (measured here)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        sink = torch.empty(sms * 8 * 256 * 8, dtype=torch.uint8, device=dev)
        peak = time_probe(ks, ks.KS_PROBE_SPLITMIX, sms * 8, 2000, sink, stream)
        achieved = 2.0 * events_per_step / (total_ms / args.steps / 1e3)
        roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gmix/s",
                    "frac": achieved / peak, "traffic": None,
                    "peak_source": "measured: the kernel's SplitMix64 mix routine in a loop with nothing else",
                    "algorithmic": f"2 SplitMix64 mixes per agent-event x {events_per_step:.4g} agent-events per launch",
                    "kernel": "paper_kernel"}
    if rank == 0:
        out = {"metric": "agent_events_per_s", "value": value, "unit": "events/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
               "data": "synthetic",
               "config": {"workload": args.workload, "M": int(w["M"]), "L": int(w["L"]), "A": int(w["A"]), "S": S,
                          "model": "the paper's agents (tick-aggregated book)", "engine": args.engine,
                          "launch": "one thread per market, one launch per step" if naive else ens.get_launch(),
                          "l2": ("book rows in global memory, read and written every step (L2-resident at "
                                 "this size)" if naive else
                                 "book state resident on chip; 1 MiB of global state per 256 markets")},
               "e2e": {"value": world * events_per_step * args.e2e_steps / e2e_s, "unit": "events/s",
                       "h2d_bytes_per_step": 0, "d2h_bytes_per_step": nbytes},
               "gpu_launches": (2 * S if naive else 2) * args.steps, "roofline": roofline, "clocks": clocks,
               "paper_context": {"value": None if naive else PAPER_PEAK.get((int(w["M"]), int(w["A"]))),
                                 "hardware": "RTX 5090 (sm_120), Table III"}}
        print(json.dumps(out), flush=True)
    ens.close()
    sharding.finalize()
    return 0


def run_cda(args, w, rank, world, dev):
    """The continuous double auction as the main workload (``--workload
    cda_8192``): same timing rules; the end-to-end leg reads the state back."""
    import torch

    from paper_2606_21784_gb300 import kineticsim as ks
    from paper_2606_21784_gb300 import sharding
    ens = ks.CdaEnsemble(w)
    S = int(w["S"])
    events_per_step = float(w["M"]) * w["A"] * S
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ens.step(S, stream)
    torch.cuda.synchronize()
    sharding.barrier()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    t0e = torch.cuda.Event(enable_timing=True)
    t1e = torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    for _ in range(args.steps):
        ens.step(S, stream)
    t1e.record(stream)
    torch.cuda.synchronize()
    sharding.barrier()
    clocks = sampler.stop()
    total_ms = sharding.max_over_ranks(t0e.elapsed_time(t1e), dev)
    value = world * events_per_step * args.steps / (total_ms / 1e3)
    if ens.sync(timeout_ms=600_000) != ks.KS_OK:
        raise RuntimeError("CDA ensemble reported a device error")
    fields = ["order", "inventory", "cash", "next", "last_tick", "fills", "sum_volume"]
    ens.step(S, stream)
    ens.read_state(fields, stream)
    t0 = time.perf_counter()
    nbytes = 0
    for _ in range(args.e2e_steps):
        ens.step(S, stream)
        st = ens.read_state(fields, stream)
        nbytes = sum(a.nbytes for a in st.values())
    e2e_s = sharding.max_over_ranks(time.perf_counter() - t0, dev)
    if rank == 0:
        out = {"metric": "agent_events_per_s", "value": value, "unit": "events/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
               "data": "synthetic",
               "config": {"workload": args.workload, "M": int(w["M"]), "L": int(w["L"]), "A": int(w["A"]), "S": S,
                          "model": "continuous double auction, the configuration's agents",
                          "l2": "book resident on chip; state read and written once per launch"},
               "e2e": {"value": world * events_per_step * args.e2e_steps / e2e_s, "unit": "events/s",
                       "h2d_bytes_per_step": 0, "d2h_bytes_per_step": nbytes},
               "gpu_launches": 2 * args.steps, "roofline": cda_roofline(events_per_step, total_ms / args.steps),
               "clocks": clocks}
        print(json.dumps(out), flush=True)
    ens.close()
    sharding.finalize()
    return 0


def cda_roofline(events_per_launch, launch_ms):
    """The CDA kernel against the ALU roof of its draws: one Philox block (20
    wide products) per agent-event, the peak derived as for the plain line at
    the nominal 32 products/clk/SM.  The fraction is small by construction:
    the kernel waits on the dependent shared-memory accesses of the serial
    matching (one lane per market), not on a pipe."""
    achieved = PHILOX_MULW_PER_EVENT * events_per_launch / (launch_ms / 1e3) / 1e12
    peak = SM_COUNT_NOMINAL * 32 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tproducts/s", "frac": achieved / peak,
            "traffic": None, "kernel": "cda_kernel", "launch_ms": launch_ms,
            "algorithmic": f"{PHILOX_MULW_PER_EVENT} 32x32->64 products per agent-event x "
                           f"{events_per_launch:.4g} agent-events per launch",
            "peak_source": f"derived: {SM_COUNT_NOMINAL} SMs x 32 products/clk/SM x {SM_MAX_MHZ_NOMINAL:.0f} MHz",
            "note": "latency-bound: the matching is a chain of dependent shared-memory accesses on one lane per "
                    "market; issue slots 55% busy in the ncu capture"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
