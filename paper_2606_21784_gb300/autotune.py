"""Autotuner of the persistent kernels' launch shapes.

Plain kernel: times every compiled (threads, agents/thread, register cap)
candidate that covers the market size on the real ensemble and keeps the
fastest.

Batched kernel: splits the ensemble into power-of-two (L, A) buckets; for each
bucket and each CTA size (512, 1024) it times every compiled (group threads,
agents/thread) shape that covers the bucket on a sample of the bucket's own
markets, keeps the fastest per bucket, then picks the CTA size whose plan has
the smallest estimated total time.  Markets per CTA follow from the group
size and the shared-memory fit; the tick tile is L / group threads.

Results never change simulation outputs (only speed).  Plans are cached per
device and ensemble shape in ``_tune_cache.json`` next to this file.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import kineticsim as ks

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json")


def _cache_load():
    try:
        return json.load(open(_CACHE))
    except (OSError, ValueError):
        return {}


def _cache_store(key, value):
    c = _cache_load()
    c[key] = value
    tmp = _CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE)


def _device_tag():
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}:{p.multi_processor_count}"


def _time_steps(ens, steps):
    import torch
    ens.step(max(1, steps // 4))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    ens.step(steps)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def _pow2(x):
    return 1 << max(0, int(np.ceil(np.log2(max(int(x), 1)))))


# compiled policy-capable shapes: (threads, agents per thread, register cap classes)
POLICY_SHAPES = ((128, 16, (0, 1)), (256, 8, (0, 1)), (256, 16, (0, 1)), (512, 4, (0,)), (512, 8, (0,)), (512, 16, (0,)),
                 (1024, 8, (0,)), (1024, 16, (0,)))


def plain_candidates(A, policy: bool = False):
    out = []
    if policy:
        return [dict(threads=nt, agents_per_thread=ak, reg_cap=rc) for nt, ak, rcs in POLICY_SHAPES
                for rc in rcs if A <= nt * ak <= 4 * max(A, 128)]
    for nt in (128, 256, 512, 1024):
        for ak in (1, 2, 4, 8, 16):
            if nt * ak < A or nt * ak > 4 * max(A, 32):
                continue
            # register-cap classes 1 and 2 change nothing for 512- and 1024-thread CTAs,
            # class 3 (64 registers) only for them; shapes that are not compiled are
            # skipped when set_launch refuses them
            for rc in ((0, 1, 2) if nt <= 256 else (0, 3)):
                out.append(dict(threads=nt, agents_per_thread=ak, reg_cap=rc))
    return out


def tune_plain(w: dict, steps: int = 40, use_cache: bool = True, verbose: bool = False, mlp_params=None) -> dict:
    """Best plain-kernel launch for a uniform workload dict; applies nothing.
    With mlp_params (policy agents), the policy-capable shapes are timed."""
    M, L, A = int(w["M"]), int(w["L"]), int(w["A"])
    policy = mlp_params is not None and int(w["params"].get("mlp_pct", 0)) > 0
    key = f"plain|{_device_tag()}|L{L}|A{A}|M{M}|carry{w['params']['carry_book']}|policy{int(policy)}"
    if use_cache:
        c = _cache_load().get(key)
        if c:
            return c
    ens = ks.Ensemble(w, mlp_params=mlp_params)
    events = float(M) * A * steps
    best = None
    for cand in plain_candidates(A, policy):
        try:
            ens.set_launch(**cand)
        except ks.KsError:
            continue
        rate = events / _time_steps(ens, steps)
        if verbose:
            print("plain", cand, f"{rate:.3e}")
        if best is None or rate > best[0]:
            best = (rate, cand)
    ens.close()
    out = dict(best[1], events_per_s=best[0])
    _cache_store(key, out)
    return out


def buckets_of(L, A):
    """Power-of-two (L, A) classes of an ensemble: {(Lc, Ac): [market indices]}."""
    out = {}
    for m, (l, a) in enumerate(zip(L, A)):
        out.setdefault((max(32, _pow2(l)), max(32, _pow2(a))), []).append(m)
    return out


def tune_batched(w: dict, L=None, A=None, steps: int = 20, max_sample: int = 1216, use_cache: bool = True,
                 verbose: bool = False, check_default: bool = True) -> dict:
    """Returns {"cta_threads": nt, "buckets": [(L_max, A_max, gt, ak), ...]} for an uneven workload,
    or buckets None when the library's default plan ran the whole ensemble faster."""
    from . import workloads
    if L is None or A is None:
        L, A = workloads.sizes(w)
    L = np.asarray(L, np.int32)
    A = np.asarray(A, np.int32)
    h = hashlib.sha256(L.tobytes() + A.tobytes()).hexdigest()[:16]
    key = f"batched|{_device_tag()}|{h}|carry{w['params']['carry_book']}|vsdefault{int(check_default)}"
    if use_cache:
        c = _cache_load().get(key)
        if c:
            return c
    groups = buckets_of(L, A)
    rng = np.random.default_rng(0)
    plans = {}
    for nt in (512, 1024):
        variants = ks.ks_batch_variants(nt)
        total = 0.0
        chosen = []
        for (Lc, Ac), members in sorted(groups.items()):
            members = np.asarray(members)
            if len(members) > max_sample:
                members = np.sort(rng.choice(members, max_sample, replace=False))
            sub = dict(w, M=len(members), market_base=0)
            cands = [(g, k) for g, k in variants if Ac <= g * k <= 4 * Ac]
            best = None
            ens = ks.Ensemble(sub, L=L[members], A=A[members])
            ev = float(A[members].astype(np.int64).sum()) * steps
            for g, k in cands:
                try:
                    ens.set_batch_plan(nt, [(Lc, Ac, g, k)])
                except ks.KsError:
                    continue
                rate = ev / _time_steps(ens, steps)
                if verbose:
                    print("batched", nt, (Lc, Ac), (g, k), f"{rate:.3e}")
                if best is None or rate > best[0]:
                    best = (rate, g, k)
            ens.close()
            if best is None:
                total = float("inf")
                break
            bucket_events = float(A[groups[(Lc, Ac)]].astype(np.int64).sum())
            total += bucket_events / best[0]
            chosen.append((int(Lc), int(Ac), int(best[1]), int(best[2])))
        plans[nt] = (total, chosen)
    nt = min(plans, key=lambda k: plans[k][0])
    out = {"cta_threads": nt, "buckets": plans[nt][1], "estimated_s_per_step": plans[nt][0]}
    # A bucket timed alone fills the GPU poorly when its markets are few or
    # small, so the composed plan is checked against the library's default
    # plan on the whole ensemble; buckets None means "keep the default".
    if not check_default:
        _cache_store(key, out)
        return out
    full = dict(w, M=len(L), market_base=0)
    ev = float(A.astype(np.int64).sum()) * steps
    ens = ks.Ensemble(full, L=L, A=A)
    default_rate = ev / _time_steps(ens, steps)
    default_nt = int(ens.batch_info()["cta_threads"])
    try:
        ens.set_batch_plan(nt, out["buckets"])
        tuned_rate = ev / _time_steps(ens, steps)
    except ks.KsError:
        tuned_rate = 0.0
    ens.close()
    if verbose:
        print("batched whole ensemble: default", f"{default_rate:.3e}", "tuned", f"{tuned_rate:.3e}")
    if default_rate >= tuned_rate:
        out = {"cta_threads": default_nt, "buckets": None, "estimated_s_per_step": plans[nt][0],
               "kept_default": True}
    _cache_store(key, out)
    return out


# compiled shapes of the paper-agent kernel: (threads per market, agents per thread, min resident CTAs)
PAPER_SHAPES = ((32, 1, 1), (32, 2, 1), (32, 4, 1), (32, 1, 8), (32, 2, 8), (32, 8, 1), (32, 8, 6), (32, 16, 1),
                (32, 32, 1), (128, 1, 1), (128, 2, 1), (128, 4, 1),
                (128, 8, 1), (128, 16, 1), (128, 1, 8), (128, 2, 8), (128, 4, 6), (128, 8, 6), (256, 1, 1),
                (256, 2, 1), (256, 4, 1), (256, 8, 1), (256, 16, 1), (512, 16, 1), (1024, 16, 1),
                (16, 1, 1), (16, 2, 1), (16, 4, 1), (16, 2, 8), (16, 4, 8), (64, 4, 1), (64, 8, 1))


def tune_paper(w: dict, steps: int = 100, use_cache: bool = True, verbose: bool = False) -> dict:
    """Best launch of the paper-agent kernel for workload dict ``w``; applies nothing."""
    M, L, A = int(w["M"]), int(w["L"]), int(w["A"])
    key = f"paper|{_device_tag()}|L{L}|A{A}|M{M}"
    if use_cache:
        c = _cache_load().get(key)
        if c:
            return c
    ens = ks.PaperEnsemble(w)
    best = None
    for nt, ak, mc in PAPER_SHAPES:
        if nt * ak < A or nt * ak > 8 * max(A, 128):
            continue
        try:
            ens.set_launch(nt, ak, mc)
        except ks.KsError:
            continue
        rate = float(M) * A * steps / _time_steps(ens, steps)
        if verbose:
            print("paper", (nt, ak, mc), f"{rate:.3e}")
        if best is None or rate > best[0]:
            best = (rate, dict(threads=nt, agents_per_thread=ak, min_ctas=mc))
    ens.close()
    out = dict(best[1], events_per_s=best[0])
    _cache_store(key, out)
    return out


def apply(ens, w: dict, use_cache: bool = True, verbose: bool = False) -> dict:
    """Tunes and applies the launch of an Ensemble (or PaperEnsemble) built from workload dict ``w``."""
    if isinstance(ens, ks.PaperEnsemble):
        best = tune_paper(w, use_cache=use_cache, verbose=verbose)
        ens.set_launch(best["threads"], best["agents_per_thread"], best["min_ctas"])
        return best
    if ens.batch_info()["batched"]:
        plan = tune_batched(w, ens.L, ens.A, use_cache=use_cache, verbose=verbose)
        if plan["buckets"] is not None:
            ens.set_batch_plan(plan["cta_threads"], plan["buckets"])
        return plan
    best = tune_plain(w, use_cache=use_cache, verbose=verbose, mlp_params=getattr(ens, "mlp_params", None))
    ens.set_launch(best["threads"], best["agents_per_thread"], reg_cap=best["reg_cap"])
    return best
