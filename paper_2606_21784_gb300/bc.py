"""Behaviour cloning of the agent policy from the rule-based simulator.

1. ``generate``: runs the rule-based 8192-market configuration (L=1024,
   A=4096, 60/20/20 agent mix, carried book) with seed 7 on the GPU and
   records the new orders of the first ``record_agents`` agents of every
   market (features and action), in a canonical order, ``n_pairs`` of them.
2. ``train``: minibatch Adam on the records with the library's hand-written
   forward/backward kernels (``ks_bc_grad``, ``ks_adam_step``).
3. ``evaluate`` / ``action_match``: held-out loss, and agreement of the
   policy's most likely side and offset with the rule agents' choices.
4. ``export``: the BF16 blob the step loop reads.

Python only orchestrates: every forward, backward and update runs in the
CUDA kernels of the library.
"""
from __future__ import annotations

import math

import numpy as np

from . import kineticsim as ks
from . import workloads

DECISIONS_PER_AGENT_STEP = 0.25  # lower bound of the rule agents' order rate (measured ~0.29)


def canonical_order(records):
    """The records sorted lexicographically by their words (first word most
    significant): one order for one multiset of records, whatever order the
    kernels appended them in."""
    import torch
    idx = torch.arange(records.shape[0], device=records.device)
    for j in reversed(range(records.shape[1])):
        _, o = torch.sort(records[idx, j], stable=True)
        idx = idx[o]
    return records[idx].contiguous()


def generate(n_pairs: int = 20_000_000, seed: int = 7, record_agents: int = 64, steps: int = 2000,
             markets: int | None = None):
    """Records of rule decisions (device int32 [n, 22]) and the workload used.

    The kernels append records in completion order, so the run keeps every
    record (a second run with the exact capacity when the first fills up),
    puts them in canonical order and, when there are more than ``n_pairs``,
    keeps ``n_pairs`` of them chosen by a generator seeded with ``seed``: the
    same arguments give the same records, and so the same trained network."""
    import torch
    w = workloads.workload("plain_mix_8192", seed=seed)
    if markets is None:
        markets = int(math.ceil(n_pairs / (DECISIONS_PER_AGENT_STEP * record_agents * steps)))
    w["M"] = markets
    w["S"] = steps
    capacity = int(n_pairs * 1.5) + 1024
    for _ in range(2):
        ens = ks.Ensemble(w)
        cap = ens.set_capture(record_agents=record_agents, record_capacity=capacity)
        ens.step(steps)
        if ens.sync(timeout_ms=600_000) != ks.KS_OK:
            raise RuntimeError("data generation run reported a device error")
        torch.cuda.synchronize()
        count = int(cap["record_count"].item())
        ens.close()
        if count <= capacity:
            break
        capacity = count
    rec = canonical_order(cap["records"][:count])
    del cap
    if count > n_pairs:
        g = torch.Generator(device=rec.device).manual_seed(seed)
        keep = torch.randperm(count, generator=g, device=rec.device)[:n_pairs].sort().values
        rec = rec[keep].contiguous()
    return rec, w


def init_params(seed: int = 0, device="cuda"):
    """He-normal weights, zero biases (log-quantity bias at log 30)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    parts = []
    for fan_out, fan_in in ((64, 32), (64, 64), (37, 64)):
        parts.append(torch.randn(fan_out * fan_in, generator=g) * math.sqrt(2.0 / fan_in))
        b = torch.zeros(fan_out)
        if fan_out == 37:
            b[36] = math.log(30.0)
        parts.append(b)
    return torch.cat(parts).float().to(device).contiguous()


def marginal_params(records, device="cuda"):
    """Zero weights; biases = log label frequencies and the mean log-quantity:
    the best policy that ignores its inputs."""
    import torch
    r = records.long()
    side = torch.bincount(r[:, 18], minlength=3).double() + 1e-3
    off = torch.bincount(r[:, 19], minlength=33).double() + 1e-3
    b3 = torch.cat([torch.log(side / side.sum()), torch.log(off / off.sum()),
                    torch.log(r[:, 20].double()).mean().reshape(1)])
    p = torch.zeros(ks.KS_MLP_NPARAM, dtype=torch.float64)
    p[-37:] = b3.cpu()
    return p.float().to(device).contiguous()


def evaluate(params, records, A: int, chunk: int = 1 << 20) -> float:
    """Mean loss of ``params`` over ``records``."""
    import torch
    n = records.shape[0]
    grad = torch.zeros(ks.KS_MLP_NPARAM, dtype=torch.float32, device=params.device)
    loss = torch.zeros(1, dtype=torch.float32, device=params.device)
    ws = None
    for i in range(0, n, chunk):
        ws = ks.ks_bc_grad(params, records[i:i + chunk].contiguous(), A, grad, loss, 1.0 / n, workspace=ws)
    torch.cuda.synchronize()
    return float(loss.item())


def features(records, A: int):
    """Normalised policy inputs of records (device float32 [n, 32])."""
    import torch
    r = records.float()
    X = torch.zeros((records.shape[0], 32), dtype=torch.float32, device=records.device)
    X[:, :8] = r[:, :8] / 8.0
    X[:, 8] = r[:, 8] / 256.0
    X[:, 9] = r[:, 9] / (8.0 * A)
    X[:, 10:18] = r[:, 10:18] / (4.0 * A)
    return X


def action_match(blob, records, A: int) -> dict:
    """Agreement of the policy's most likely side / offset with the recorded actions
    (logits from the tensor-core forward)."""
    Z, err = ks.ks_mlp_forward(blob, features(records, A))
    side = Z[:, :3].argmax(1)
    off = Z[:, 3:36].argmax(1)
    r = records.long()
    return {"side": float((side == r[:, 18]).float().mean()), "offset": float((off == r[:, 19]).float().mean()),
            "error_word": int(err.item())}


def train(records, A: int, epochs: int = 2, batch: int = 16384, lr: float = 2e-3, val_frac: float = 0.02,
          seed: int = 0, params=None, log=None):
    """Adam on the records; returns (params, history)."""
    import torch
    dev = records.device
    n = records.shape[0]
    g = torch.Generator(device=dev).manual_seed(seed)
    perm = torch.randperm(n, generator=g, device=dev)
    n_val = max(1, int(n * val_frac))
    val = records[perm[:n_val]].contiguous()
    tr_idx = perm[n_val:]
    params = init_params(seed, dev) if params is None else params.clone()
    grad = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    ws = torch.empty(max(ks.ks_bc_workspace_size(batch), 1), dtype=torch.uint8, device=dev)
    hist = {"val_loss": [evaluate(params, val, A)], "train_loss": []}
    step = 0
    for ep in range(epochs):
        order = tr_idx[torch.randperm(tr_idx.shape[0], generator=g, device=dev)]
        loss.zero_()
        seen = 0
        for i in range(0, order.shape[0], batch):
            idx = order[i:i + batch]
            bs = idx.shape[0]
            ks.ks_bc_grad(params, records[idx].contiguous(), A, grad, loss, 1.0 / bs, workspace=ws)
            step += 1
            ks.ks_adam_step(params, grad, m, v, step, lr)
            seen += 1
        torch.cuda.synchronize()
        hist["train_loss"].append(float(loss.item()) / max(seen, 1))
        hist["val_loss"].append(evaluate(params, val, A))
        if log:
            log(f"epoch {ep}: train {hist['train_loss'][-1]:.4f} val {hist['val_loss'][-1]:.4f}")
    return params, hist, val


def export(params):
    return ks.ks_mlp_export(params)


def main(argv=None):
    """Full pipeline: 20M pairs from the seed-7 rule-based run, training, report."""
    import argparse
    import json
    import time

    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=20_000_000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)
    t0 = time.time()
    rec, w = generate(a.pairs)
    t1 = time.time()
    params, hist, val = train(rec, w["A"], epochs=a.epochs, batch=a.batch, lr=a.lr, log=print)
    torch.cuda.synchronize()
    t2 = time.time()
    blob = export(params)
    rep = {"pairs": int(rec.shape[0]), "markets": w["M"], "generate_s": t1 - t0, "train_s": t2 - t1,
           "history": hist, "held_out_loss": {"trained": evaluate(params, val, w["A"]),
                                              "marginal": evaluate(marginal_params(rec), val, w["A"]),
                                              "untrained": evaluate(init_params(0), val, w["A"])},
           "action_match": {"trained": action_match(blob, val, w["A"]),
                            "marginal": action_match(export(marginal_params(rec)), val, w["A"])}}
    print(json.dumps(rep))
    if a.out:
        with open(a.out, "wb") as f:
            f.write(blob.cpu().numpy().tobytes())
    return rep


if __name__ == "__main__":
    main()
