"""ctypes binding of ``libkineticsim.so`` (the C ABI of ``include/kineticsim.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of the library.  PyTorch provides device memory and streams.  There is
no fallback: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

KS_OK = 0
KS_ERR_INVALID_ARG = 1
KS_ERR_WORKSPACE_TOO_SMALL = 2
KS_ERR_CUDA = 3
KS_ERR_UNSUPPORTED = 4
KS_ERR_DEVICE_FAULT = 5
KS_ERR_TIMEOUT = 6
KS_HISTORY = 9

_STATUS = {0: "KS_OK", 1: "KS_ERR_INVALID_ARG", 2: "KS_ERR_WORKSPACE_TOO_SMALL", 3: "KS_ERR_CUDA",
           4: "KS_ERR_UNSUPPORTED", 5: "KS_ERR_DEVICE_FAULT", 6: "KS_ERR_TIMEOUT"}

# every entry point declared in include/kineticsim.h
EXPORTS = ("ks_workspace_size", "ks_create_ensemble", "ks_step_n", "ks_read_state", "ks_write_state",
           "ks_sync", "ks_error_word", "ks_set_launch", "ks_get_launch", "ks_destroy", "ks_status_string",
           "ks_last_error", "ks_version", "ks_probe", "ks_probe_state_io", "ks_set_batch_plan",
           "ks_get_batch_info", "ks_batch_variants", "ks_mlp_forward", "ks_set_capture", "ks_bc_grad",
           "ks_bc_workspace_size",
           "ks_adam_step", "ks_mlp_export", "ks_paper_workspace_size", "ks_paper_create", "ks_paper_step_n",
           "ks_paper_step_n_naive", "ks_paper_read_state", "ks_paper_set_launch", "ks_paper_get_launch",
           "ks_paper_sync", "ks_paper_destroy", "ks_cda_workspace_size", "ks_cda_create", "ks_cda_step_n",
           "ks_cda_read_state", "ks_cda_sync", "ks_cda_destroy")
KS_MLP_NPARAM = 8677

KS_RECORD_WORDS = 22
KS_DECISION_PASS = 0x01000000
KS_DECISION_NONE = 0xFFFFFFFF

KS_MLP_PARAM_BYTES = 17696
MLP_IN, MLP_H, MLP_OUT = 32, 64, 37


class KsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)} {detail}".strip())


class ks_config(ctypes.Structure):
    _fields_ = [
        ("n_markets", ctypes.c_uint32),
        ("market_base", ctypes.c_uint32),
        ("L", ctypes.POINTER(ctypes.c_int32)),
        ("A", ctypes.POINTER(ctypes.c_int32)),
        ("L_all", ctypes.c_int32),
        ("A_all", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("carry_book", ctypes.c_int32),
        ("cancel_thresh_q32", ctypes.c_uint32),
        ("mix_pct", ctypes.c_uint32 * 3),
        ("zi_offset", ctypes.c_int32),
        ("zi_qmax", ctypes.c_int32),
        ("mom_lookback", ctypes.c_int32),
        ("mom_offset_max", ctypes.c_int32),
        ("mr_offset_max", ctypes.c_int32),
        ("rb_qmax", ctypes.c_int32),
        ("mlp_pct", ctypes.c_uint32),
        ("mlp_params", ctypes.c_void_p),
        ("tie_rule", ctypes.c_int32),
        ("trace_markets", ctypes.c_uint32),
        ("trace_steps", ctypes.c_uint32),
    ]


class ks_state_view(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "order", "inventory", "cash", "last_tick", "history", "fundamental", "trades", "last_volume",
        "sum_price", "sum_volume", "trace_hash", "step", "trace")]


class ks_launch(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("agents_per_thread", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("aggregate", ctypes.c_int32), ("reg_cap", ctypes.c_int32)]


class ks_bucket(ctypes.Structure):
    _fields_ = [("L_max", ctypes.c_int32), ("A_max", ctypes.c_int32), ("group_threads", ctypes.c_int32),
                ("agents_per_thread", ctypes.c_int32)]


class ks_capture(ctypes.Structure):
    _fields_ = [("records", ctypes.c_void_p), ("record_capacity", ctypes.c_uint64),
                ("record_agents", ctypes.c_uint32), ("pad_", ctypes.c_uint32),
                ("record_count", ctypes.c_void_p), ("decisions", ctypes.c_void_p),
                ("policy_count", ctypes.c_void_p), ("logits", ctypes.c_void_p)]


class ks_batch_info(ctypes.Structure):
    _fields_ = [("batched", ctypes.c_int32), ("cta_threads", ctypes.c_int32), ("n_items", ctypes.c_int32),
                ("n_buckets", ctypes.c_int32), ("grid", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int64)]


class ks_paper_config(ctypes.Structure):
    _fields_ = [("n_markets", ctypes.c_uint32), ("market_base", ctypes.c_uint32), ("L", ctypes.c_int32),
                ("A", ctypes.c_int32), ("seed", ctypes.c_uint64), ("noise_halfwidth", ctypes.c_int32),
                ("p_mkt_q32", ctypes.c_uint32), ("qmax", ctypes.c_int32), ("maker_half_spread", ctypes.c_int32),
                ("mom_pct", ctypes.c_uint32), ("maker_pct", ctypes.c_uint32), ("tie_rule", ctypes.c_int32),
                ("trace_markets", ctypes.c_uint32), ("trace_steps", ctypes.c_uint32), ("window", ctypes.c_int32)]


class ks_cda_config(ctypes.Structure):
    _fields_ = [("n_markets", ctypes.c_uint32), ("market_base", ctypes.c_uint32), ("L", ctypes.c_int32),
                ("A", ctypes.c_int32), ("seed", ctypes.c_uint64), ("cancel_thresh_q32", ctypes.c_uint32),
                ("mix_pct", ctypes.c_uint32 * 3), ("zi_offset", ctypes.c_int32), ("zi_qmax", ctypes.c_int32),
                ("mom_lookback", ctypes.c_int32), ("mom_offset_max", ctypes.c_int32),
                ("mr_offset_max", ctypes.c_int32), ("rb_qmax", ctypes.c_int32), ("trace_markets", ctypes.c_uint32),
                ("trace_steps", ctypes.c_uint32)]


class ks_cda_state_view(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "order", "inventory", "cash", "next", "last_tick", "history", "fundamental", "fills", "last_volume",
        "traded_value", "sum_volume", "trace_hash", "step", "trace")]


class ks_paper_state_view(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "bid", "ask", "last_tick", "mid2", "trades", "last_volume", "sum_price", "sum_volume", "trace_hash",
        "step", "trace", "window_base")]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if needed).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    sig = {
        "ks_workspace_size": ([P(ks_config), P(ctypes.c_size_t)], ctypes.c_int),
        "ks_create_ensemble": ([P(ks_config), vp, ctypes.c_size_t, vp, P(vp)], ctypes.c_int),
        "ks_step_n": ([vp, ctypes.c_uint32, vp], ctypes.c_int),
        "ks_read_state": ([vp, P(ks_state_view), vp], ctypes.c_int),
        "ks_write_state": ([vp, P(ks_state_view), vp], ctypes.c_int),
        "ks_sync": ([vp, vp, ctypes.c_uint32], ctypes.c_int),
        "ks_error_word": ([vp, vp, P(ctypes.c_uint32)], ctypes.c_int),
        "ks_set_launch": ([vp, P(ks_launch)], ctypes.c_int),
        "ks_get_launch": ([vp, P(ks_launch)], ctypes.c_int),
        "ks_destroy": ([vp], ctypes.c_int),
        "ks_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "ks_last_error": ([], ctypes.c_char_p),
        "ks_version": ([], ctypes.c_uint32),
        "ks_probe": ([ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, vp, vp, P(ctypes.c_double)], ctypes.c_int),
        "ks_probe_state_io": ([vp, vp, P(ctypes.c_double)], ctypes.c_int),
        "ks_set_batch_plan": ([vp, ctypes.c_int32, P(ks_bucket), ctypes.c_int32, vp], ctypes.c_int),
        "ks_get_batch_info": ([vp, P(ks_batch_info)], ctypes.c_int),
        "ks_batch_variants": ([ctypes.c_int32, P(ctypes.c_int32), ctypes.c_int32, P(ctypes.c_int32)], ctypes.c_int),
        "ks_mlp_forward": ([vp, vp, ctypes.c_int64, vp, vp, vp], ctypes.c_int),
        "ks_set_capture": ([vp, P(ks_capture)], ctypes.c_int),
        "ks_bc_workspace_size": ([ctypes.c_int64, P(ctypes.c_size_t)], ctypes.c_int),
        "ks_bc_grad": ([vp, vp, ctypes.c_int64, ctypes.c_int32, vp, vp, ctypes.c_float, vp, ctypes.c_size_t, vp],
                       ctypes.c_int),
        "ks_adam_step": ([vp, vp, vp, vp, ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, vp], ctypes.c_int),
        "ks_mlp_export": ([vp, vp, vp], ctypes.c_int),
        "ks_paper_workspace_size": ([P(ks_paper_config), P(ctypes.c_size_t)], ctypes.c_int),
        "ks_paper_create": ([P(ks_paper_config), vp, ctypes.c_size_t, vp, P(vp)], ctypes.c_int),
        "ks_paper_step_n": ([vp, ctypes.c_uint32, vp], ctypes.c_int),
        "ks_paper_step_n_naive": ([vp, ctypes.c_uint32, vp], ctypes.c_int),
        "ks_paper_read_state": ([vp, P(ks_paper_state_view), vp], ctypes.c_int),
        "ks_paper_set_launch": ([vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
        "ks_paper_get_launch": ([vp, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)], ctypes.c_int),
        "ks_paper_sync": ([vp, vp, ctypes.c_uint32], ctypes.c_int),
        "ks_paper_destroy": ([vp], ctypes.c_int),
        "ks_cda_workspace_size": ([P(ks_cda_config), P(ctypes.c_size_t)], ctypes.c_int),
        "ks_cda_create": ([P(ks_cda_config), vp, ctypes.c_size_t, vp, P(vp)], ctypes.c_int),
        "ks_cda_step_n": ([vp, ctypes.c_uint32, vp], ctypes.c_int),
        "ks_cda_read_state": ([vp, P(ks_cda_state_view), vp], ctypes.c_int),
        "ks_cda_sync": ([vp, vp, ctypes.c_uint32], ctypes.c_int),
        "ks_cda_destroy": ([vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != KS_OK:
        detail = load().ks_last_error()
        raise KsError(rc, where, detail.decode() if detail else "")


def _stream_ptr(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def make_config(w: dict, trace_markets: int = 0, trace_steps: int = 0, L=None, A=None, mlp_params=None):
    """ks_config from a workload dict (see ``workloads``).  Returns (config, keepalive)."""
    from . import workloads
    p = w["params"]
    c = ks_config()
    M = int(w["M"])
    c.n_markets = M
    c.market_base = int(w.get("market_base", 0))
    keep = []
    if L is None or A is None:
        L, A = workloads.sizes(w)
    L = np.ascontiguousarray(L, dtype=np.int32)
    A = np.ascontiguousarray(A, dtype=np.int32)
    uniform = bool(np.all(L == L[0]) and np.all(A == A[0]))
    if uniform:
        c.L_all, c.A_all = int(L[0]), int(A[0])
    else:
        c.L = L.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        c.A = A.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        keep += [L, A]
    c.seed = int(p["seed"])
    c.carry_book = int(p["carry_book"])
    c.cancel_thresh_q32 = int(p["cancel_thresh_q32"])
    for i in range(3):
        c.mix_pct[i] = int(p["mix_pct"][i])
    c.zi_offset = int(p["zi_offset"])
    c.zi_qmax = int(p["zi_qmax"])
    c.mom_lookback = int(p["mom_lookback"])
    c.mom_offset_max = int(p["mom_offset_max"])
    c.mr_offset_max = int(p["mr_offset_max"])
    c.rb_qmax = int(p["rb_qmax"])
    c.mlp_pct = int(p.get("mlp_pct", 0))
    c.mlp_params = mlp_params.data_ptr() if mlp_params is not None else None
    c.tie_rule = int(p.get("tie_rule", 0))
    c.trace_markets = int(trace_markets)
    c.trace_steps = int(trace_steps)
    return c, (keep, L, A)


# ---------------------------------------------------------------------------
# Thin wrappers with the C names
# ---------------------------------------------------------------------------
def ks_workspace_size(cfg: ks_config) -> int:
    n = ctypes.c_size_t(0)
    _check(load().ks_workspace_size(ctypes.byref(cfg), ctypes.byref(n)), "ks_workspace_size")
    return int(n.value)


def ks_create_ensemble(cfg: ks_config, workspace_ptr: int, ws_bytes: int, stream=None) -> int:
    h = ctypes.c_void_p(0)
    _check(load().ks_create_ensemble(ctypes.byref(cfg), workspace_ptr, ws_bytes, _stream_ptr(stream),
                                     ctypes.byref(h)), "ks_create_ensemble")
    return h.value


def ks_step_n(h: int, n_steps: int, stream=None):
    _check(load().ks_step_n(h, int(n_steps), _stream_ptr(stream)), "ks_step_n")


def ks_read_state(h: int, view: ks_state_view, stream=None):
    _check(load().ks_read_state(h, ctypes.byref(view), _stream_ptr(stream)), "ks_read_state")


def ks_write_state(h: int, view: ks_state_view, stream=None):
    _check(load().ks_write_state(h, ctypes.byref(view), _stream_ptr(stream)), "ks_write_state")


def ks_sync(h: int, stream=None, timeout_ms: int = 0) -> int:
    """Returns the status (KS_OK, KS_ERR_TIMEOUT or KS_ERR_DEVICE_FAULT); raises on other errors."""
    rc = load().ks_sync(h, _stream_ptr(stream), int(timeout_ms))
    if rc not in (KS_OK, KS_ERR_TIMEOUT, KS_ERR_DEVICE_FAULT):
        _check(rc, "ks_sync")
    return rc


def ks_error_word(h: int, stream=None) -> int:
    w = ctypes.c_uint32(0)
    _check(load().ks_error_word(h, _stream_ptr(stream), ctypes.byref(w)), "ks_error_word")
    return int(w.value)


def ks_set_launch(h: int, threads: int, agents_per_thread: int, ctas_per_sm: int = 0, aggregate: int = 0,
                  reg_cap: int = 0):
    l = ks_launch(threads, agents_per_thread, ctas_per_sm, aggregate, reg_cap)
    _check(load().ks_set_launch(h, ctypes.byref(l)), "ks_set_launch")


def ks_get_launch(h: int) -> dict:
    l = ks_launch()
    _check(load().ks_get_launch(h, ctypes.byref(l)), "ks_get_launch")
    return dict(threads=l.threads, agents_per_thread=l.agents_per_thread, ctas_per_sm=l.ctas_per_sm,
                aggregate=l.aggregate, reg_cap=l.reg_cap)


def ks_set_batch_plan(h: int, cta_threads: int, buckets, stream=None):
    """buckets: sequence of (L_max, A_max, group_threads, agents_per_thread)."""
    arr = (ks_bucket * len(buckets))(*[ks_bucket(*map(int, b)) for b in buckets])
    _check(load().ks_set_batch_plan(h, int(cta_threads), arr, len(buckets), _stream_ptr(stream)), "ks_set_batch_plan")


def ks_get_batch_info(h: int) -> dict:
    i = ks_batch_info()
    _check(load().ks_get_batch_info(h, ctypes.byref(i)), "ks_get_batch_info")
    return {f: getattr(i, f) for f, _ in ks_batch_info._fields_ if f != "pad_"}


def ks_batch_variants(cta_threads: int):
    n = ctypes.c_int32(0)
    _check(load().ks_batch_variants(int(cta_threads), None, 0, ctypes.byref(n)), "ks_batch_variants")
    buf = (ctypes.c_int32 * (2 * n.value))()
    _check(load().ks_batch_variants(int(cta_threads), buf, n.value, ctypes.byref(n)), "ks_batch_variants")
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(n.value)]


def pack_mlp_params(W1, b1, W2, b2, W3, b3, device="cuda"):
    """Device parameter blob of the policy (layout in kineticsim.h): BF16
    weights (rounded to nearest even from the given values), FP32 biases."""
    import torch
    blob = torch.zeros(KS_MLP_PARAM_BYTES, dtype=torch.uint8)
    off = 0
    for W in (W1, W2, W3):
        t = torch.as_tensor(np.asarray(W, np.float32)).to(torch.bfloat16).contiguous()
        b = t.view(torch.uint8).reshape(-1)
        blob[off:off + b.numel()] = b
        off += b.numel()
    for bias in (b1, b2, b3):
        t = torch.as_tensor(np.asarray(bias, np.float32)).contiguous()
        b = t.view(torch.uint8).reshape(-1)
        blob[off:off + b.numel()] = b
        off += b.numel()
    return blob.to(device)


def mlp_params_as_used(W1, b1, W2, b2, W3, b3):
    """The parameter values the kernels compute with (BF16-rounded weights, FP32 biases), as float64."""
    import torch
    out = []
    for i, a in enumerate((W1, b1, W2, b2, W3, b3)):
        t = torch.as_tensor(np.asarray(a, np.float32))
        if i % 2 == 0:
            t = t.to(torch.bfloat16).float()
        out.append(t.double().numpy())
    return out


def ks_mlp_forward(params_blob, X, err=None, stream=None):
    """Logits [n, 37] (fp32, device) of feature rows X [n, 32] (fp32, device)."""
    import torch
    X = X.contiguous()
    n = X.shape[0]
    Z = torch.empty((n, MLP_OUT), dtype=torch.float32, device=X.device)
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=X.device)
    _check(load().ks_mlp_forward(params_blob.data_ptr(), X.data_ptr(), n, Z.data_ptr(), err.data_ptr(),
                                 _stream_ptr(stream)), "ks_mlp_forward")
    return Z, err


def ks_bc_workspace_size(n: int) -> int:
    b = ctypes.c_size_t()
    _check(load().ks_bc_workspace_size(int(n), ctypes.byref(b)), "ks_bc_workspace_size")
    return int(b.value)


def ks_bc_grad(params, records, A: int, grad, loss, scale: float, workspace=None, stream=None):
    """grad += scale * dL/dparams, loss += scale * L over ``records`` (device).
    ``workspace``: a device uint8 tensor of at least ks_bc_workspace_size(n)
    bytes (allocated here when omitted)."""
    import torch
    n = int(records.shape[0])
    need = ks_bc_workspace_size(n)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=params.device)
    _check(load().ks_bc_grad(params.data_ptr(), records.data_ptr(), n, int(A), grad.data_ptr(),
                             loss.data_ptr(), float(scale), workspace.data_ptr(), workspace.numel(),
                             _stream_ptr(stream)), "ks_bc_grad")
    return workspace


def ks_adam_step(params, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().ks_adam_step(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), int(step), float(lr),
                               float(beta1), float(beta2), float(eps), _stream_ptr(stream)), "ks_adam_step")


def ks_mlp_export(params, blob=None, stream=None):
    import torch
    if blob is None:
        blob = torch.zeros(KS_MLP_PARAM_BYTES, dtype=torch.uint8, device=params.device)
    _check(load().ks_mlp_export(params.data_ptr(), blob.data_ptr(), _stream_ptr(stream)), "ks_mlp_export")
    return blob


KS_PROBE_SMEM_RED, KS_PROBE_MUL_WIDE, KS_PROBE_PHILOX, KS_PROBE_MUL_HILO, KS_PROBE_SPLITMIX = 0, 1, 2, 3, 4
KS_PROBE_WAIT_TIMEOUT = 5


def ks_probe(kind: int, blocks: int, iters: int, sink_ptr: int, stream=None) -> float:
    ops = ctypes.c_double(0)
    _check(load().ks_probe(kind, blocks, iters, sink_ptr, _stream_ptr(stream), ctypes.byref(ops)), "ks_probe")
    return float(ops.value)


def ks_probe_state_io(h: int, stream=None) -> float:
    b = ctypes.c_double(0)
    _check(load().ks_probe_state_io(h, _stream_ptr(stream), ctypes.byref(b)), "ks_probe_state_io")
    return float(b.value)


def ks_destroy(h: int):
    _check(load().ks_destroy(h), "ks_destroy")


# ---------------------------------------------------------------------------
# Ensemble: workspace owned by a torch tensor
# ---------------------------------------------------------------------------
STATE_FIELDS = {
    # name: (dtype, per) with per in {"agent", "market", "hist", "one", "trace"}
    "order": (np.uint32, "agent"),
    "inventory": (np.int32, "agent"),
    "cash": (np.int64, "agent"),
    "last_tick": (np.int32, "market"),
    "history": (np.int32, "hist"),
    "fundamental": (np.int32, "market"),
    "trades": (np.int32, "market"),
    "last_volume": (np.int32, "market"),
    "sum_price": (np.int64, "market"),
    "sum_volume": (np.int64, "market"),
    "trace_hash": (np.uint64, "market"),
    "step": (np.uint64, "one"),
    "trace": (np.int32, "trace"),
}

_TORCH_DT = {np.uint32: "int32", np.int32: "int32", np.int64: "int64", np.uint64: "int64"}


class Ensemble:
    """One ensemble on the current CUDA device.

    ``workload``: a dict from ``workloads.workload`` (M, L, A, params).  The
    device workspace is a torch uint8 tensor held by this object.
    """

    def __init__(self, workload: dict, trace_markets: int = 0, trace_steps: int = 0, stream=None, L=None, A=None,
                 mlp_params=None):
        import torch
        self.workload = workload
        self.mlp_params = mlp_params  # device blob kept alive for the kernels
        self.cfg, (self._keep, self.L, self.A) = make_config(workload, trace_markets, trace_steps, L, A, mlp_params)
        self.M = int(workload["M"])
        self.N = int(self.A.astype(np.int64).sum())
        self.offsets = np.concatenate([[0], np.cumsum(self.A.astype(np.int64))])
        self.trace_markets = int(trace_markets)
        self.trace_steps = int(trace_steps)
        self.ws_bytes = ks_workspace_size(self.cfg)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        self.handle = ks_create_ensemble(self.cfg, self.workspace.data_ptr(), self.ws_bytes, stream)

    def close(self):
        if getattr(self, "handle", None):
            ks_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int, stream=None):
        ks_step_n(self.handle, n, stream)

    def set_launch(self, threads, agents_per_thread, ctas_per_sm=0, aggregate=0, reg_cap=0):
        ks_set_launch(self.handle, threads, agents_per_thread, ctas_per_sm, aggregate, reg_cap)

    def get_launch(self):
        return ks_get_launch(self.handle)

    def set_batch_plan(self, cta_threads, buckets, stream=None):
        ks_set_batch_plan(self.handle, cta_threads, buckets, stream)

    def batch_info(self):
        return ks_get_batch_info(self.handle)

    def set_capture(self, record_agents: int = 0, record_capacity: int = 0, decisions: bool = False,
                    count_policy: bool = False, logits: bool = False):
        """Allocates capture buffers (torch, device) and enables them; returns them.
        ``logits``: FP32 [trace_steps, agents of the traced markets, 37], NaN
        where no policy decision was taken."""
        import torch
        c = ks_capture()
        self.capture = {}
        if record_agents > 0 and record_capacity > 0:
            rec = torch.zeros((record_capacity, KS_RECORD_WORDS), dtype=torch.int32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            c.records, c.record_capacity, c.record_agents, c.record_count = \
                rec.data_ptr(), record_capacity, record_agents, cnt.data_ptr()
            self.capture.update(records=rec, record_count=cnt)
        if count_policy:
            pc = torch.zeros(1, dtype=torch.int64, device="cuda")
            c.policy_count = pc.data_ptr()
            self.capture["policy_count"] = pc
        if decisions:
            n_tr = int(self.offsets[self.trace_markets])
            dec = torch.full((self.trace_steps, max(n_tr, 1)), -1, dtype=torch.int32, device="cuda")
            c.decisions = dec.data_ptr()
            self.capture["decisions"] = dec
        if logits:
            n_tr = int(self.offsets[self.trace_markets])
            z = torch.full((self.trace_steps, max(n_tr, 1), MLP_OUT), float("nan"), dtype=torch.float32,
                           device="cuda")
            c.logits = z.data_ptr()
            self.capture["logits"] = z
        _check(load().ks_set_capture(self.handle, ctypes.byref(c)), "ks_set_capture")
        return self.capture

    def records(self):
        """Recorded rule decisions so far (numpy int32 [n, 22])."""
        import torch
        torch.cuda.synchronize()
        n = min(int(self.capture["record_count"].item()), self.capture["records"].shape[0])
        return self.capture["records"][:n].cpu().numpy()

    def sync(self, timeout_ms: int = 0, stream=None) -> int:
        return ks_sync(self.handle, stream, timeout_ms)

    def _shape(self, per):
        return {"agent": (self.N,), "market": (self.M,), "hist": (self.M, KS_HISTORY), "one": (1,),
                "trace": (self.trace_markets, self.trace_steps, 2)}[per]

    def alloc_view(self, fields=None, device: bool = False, pinned: bool = False):
        """Allocate torch buffers for ``fields`` and a view pointing at them."""
        import torch
        fields = list(STATE_FIELDS) if fields is None else list(fields)
        bufs = {}
        v = ks_state_view()
        for f in fields:
            dt, per = STATE_FIELDS[f]
            shape = self._shape(per)
            t = torch.empty(shape, dtype=getattr(torch, _TORCH_DT[dt]),
                            device="cuda" if device else "cpu", pin_memory=(pinned and not device))
            bufs[f] = t
            setattr(v, f, t.data_ptr() if t.numel() else None)
        return v, bufs

    def read_state(self, fields=None, stream=None) -> dict:
        """Copy the state to host numpy arrays."""
        v, bufs = self.alloc_view(fields)
        ks_read_state(self.handle, v, stream)
        out = {}
        for f, t in bufs.items():
            dt = STATE_FIELDS[f][0]
            out[f] = t.numpy().view(dt).copy()
        return out

    def write_state(self, state: dict, stream=None):
        import torch
        v = ks_state_view()
        keep = []
        for f, arr in state.items():
            dt, per = STATE_FIELDS[f]
            a = np.ascontiguousarray(arr).view(dt).reshape(self._shape(per))
            t = torch.from_numpy(a.view(np.int64 if a.itemsize == 8 else np.int32).copy())
            keep.append(t)
            setattr(v, f, t.data_ptr() if t.numel() else None)
        ks_write_state(self.handle, v, stream)
        del keep

    def market_slice(self, m: int) -> slice:
        return slice(int(self.offsets[m]), int(self.offsets[m + 1]))


def unpack_orders(words: np.ndarray) -> dict:
    """Split order words into fields (layout documented in kineticsim.h)."""
    w = words.astype(np.uint32)
    return dict(qty=(w & 0xFF).astype(np.int32), side=((w >> 8) & 1).astype(np.int32),
                tick=((w >> 9) & 0xFFF).astype(np.int32), atype=((w >> 21) & 3).astype(np.int32),
                mlp=((w >> 23) & 1).astype(np.int32))



# ---------------------------------------------------------------------------
# The paper's own agents on a tick-aggregated book (ks_paper_*)
# ---------------------------------------------------------------------------
PAPER_STATE_FIELDS = {
    "bid": (np.int32, "book"), "ask": (np.int32, "book"), "last_tick": (np.int32, "market"),
    "mid2": (np.int32, "market"), "trades": (np.int32, "market"), "last_volume": (np.int32, "market"),
    "sum_price": (np.int64, "market"), "sum_volume": (np.int64, "market"), "trace_hash": (np.uint64, "market"),
    "step": (np.uint64, "one"), "trace": (np.int32, "trace"), "window_base": (np.int64, "market"),
}


def make_paper_config(w: dict, trace_markets: int = 0, trace_steps: int = 0) -> ks_paper_config:
    """ks_paper_config from a paper-agent workload dict (see ``workloads``)."""
    p = w["params"]
    return ks_paper_config(int(w["M"]), int(w.get("market_base", 0)), int(w["L"]), int(w["A"]),
                           int(p["seed"]) & 0xFFFFFFFFFFFFFFFF, int(p["noise_halfwidth"]), int(p["p_mkt_q32"]),
                           int(p["qmax"]), int(p["maker_half_spread"]), int(p["mom_pct"]), int(p["maker_pct"]),
                           int(p.get("tie_rule", 0)), int(trace_markets), int(trace_steps), int(p.get("window", 0)))


class PaperEnsemble:
    """Markets of the paper's own agent model on the current CUDA device; the
    workspace is a torch uint8 tensor held by this object."""

    def __init__(self, workload: dict, trace_markets: int = 0, trace_steps: int = 0, stream=None):
        import torch
        self.workload = workload
        self.cfg = make_paper_config(workload, trace_markets, trace_steps)
        self.M, self.L, self.A = int(workload["M"]), int(workload["L"]), int(workload["A"])
        self.trace_markets = min(int(trace_markets), self.M)
        self.trace_steps = int(trace_steps) if trace_markets else 0
        n = ctypes.c_size_t()
        _check(load().ks_paper_workspace_size(ctypes.byref(self.cfg), ctypes.byref(n)), "ks_paper_workspace_size")
        self.ws_bytes = n.value
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        _check(load().ks_paper_create(ctypes.byref(self.cfg), self.workspace.data_ptr(), self.ws_bytes,
                                      _stream_ptr(stream), ctypes.byref(h)), "ks_paper_create")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            load().ks_paper_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int, stream=None):
        _check(load().ks_paper_step_n(self.handle, int(n), _stream_ptr(stream)), "ks_paper_step_n")

    def step_naive(self, n: int, stream=None):
        """n steps by the naive engine (one thread per market, one launch per step)."""
        _check(load().ks_paper_step_n_naive(self.handle, int(n), _stream_ptr(stream)), "ks_paper_step_n_naive")

    def set_launch(self, threads: int, agents_per_thread: int, min_ctas: int = 1):
        _check(load().ks_paper_set_launch(self.handle, int(threads), int(agents_per_thread), int(min_ctas)),
               "ks_paper_set_launch")

    def get_launch(self) -> dict:
        t, k, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().ks_paper_get_launch(self.handle, ctypes.byref(t), ctypes.byref(k), ctypes.byref(c)),
               "ks_paper_get_launch")
        return {"threads": t.value, "agents_per_thread": k.value, "min_ctas": c.value}

    def sync(self, timeout_ms: int = 0, stream=None) -> int:
        return int(load().ks_paper_sync(self.handle, _stream_ptr(stream), int(timeout_ms)))

    def read_state(self, fields=None, stream=None) -> dict:
        """Copy the state to host numpy arrays (bid / ask as [M, L])."""
        import torch
        fields = list(PAPER_STATE_FIELDS) if fields is None else list(fields)
        shapes = {"book": (self.M, self.L), "market": (self.M,), "one": (1,),
                  "trace": (self.trace_markets, self.trace_steps, 2)}
        v = ks_paper_state_view()
        bufs = {}
        for f in fields:
            dt, per = PAPER_STATE_FIELDS[f]
            t = torch.empty(shapes[per], dtype=getattr(torch, _TORCH_DT[dt]))
            bufs[f] = t
            setattr(v, f, t.data_ptr() if t.numel() else None)
        _check(load().ks_paper_read_state(self.handle, ctypes.byref(v), _stream_ptr(stream)), "ks_paper_read_state")
        return {f: t.numpy().view(PAPER_STATE_FIELDS[f][0]).copy() for f, t in bufs.items()}


# ---------------------------------------------------------------------------
# Continuous double auction ensemble (ks_cda_*)
# ---------------------------------------------------------------------------
CDA_STATE_FIELDS = {
    "order": (np.uint32, "agent"), "inventory": (np.int32, "agent"), "cash": (np.int64, "agent"),
    "next": (np.int32, "agent"), "last_tick": (np.int32, "market"), "history": (np.int32, "hist"),
    "fundamental": (np.int32, "market"), "fills": (np.int32, "market"), "last_volume": (np.int32, "market"),
    "traded_value": (np.int64, "market"), "sum_volume": (np.int64, "market"), "trace_hash": (np.uint64, "market"),
    "step": (np.uint64, "one"), "trace": (np.int32, "trace"),
}


def make_cda_config(w: dict, trace_markets: int = 0, trace_steps: int = 0) -> ks_cda_config:
    """ks_cda_config from a workload dict with uniform L and A (see ``workloads``)."""
    p = w["params"]
    c = ks_cda_config()
    c.n_markets, c.market_base, c.L, c.A = int(w["M"]), int(w.get("market_base", 0)), int(w["L"]), int(w["A"])
    c.seed = int(p["seed"]) & 0xFFFFFFFFFFFFFFFF
    c.cancel_thresh_q32 = int(p["cancel_thresh_q32"])
    for i in range(3):
        c.mix_pct[i] = int(p["mix_pct"][i])
    c.zi_offset, c.zi_qmax = int(p["zi_offset"]), int(p["zi_qmax"])
    c.mom_lookback, c.mom_offset_max = int(p["mom_lookback"]), int(p["mom_offset_max"])
    c.mr_offset_max, c.rb_qmax = int(p["mr_offset_max"]), int(p["rb_qmax"])
    c.trace_markets, c.trace_steps = int(trace_markets), int(trace_steps) if trace_markets else 0
    return c


class CdaEnsemble:
    """Markets of the continuous double auction on the current CUDA device; the
    workspace is a torch uint8 tensor held by this object."""

    def __init__(self, workload: dict, trace_markets: int = 0, trace_steps: int = 0, stream=None):
        import torch
        self.workload = workload
        self.cfg = make_cda_config(workload, trace_markets, trace_steps)
        self.M, self.L, self.A = int(workload["M"]), int(workload["L"]), int(workload["A"])
        self.trace_markets = int(self.cfg.trace_markets)
        self.trace_steps = int(self.cfg.trace_steps)
        n = ctypes.c_size_t()
        _check(load().ks_cda_workspace_size(ctypes.byref(self.cfg), ctypes.byref(n)), "ks_cda_workspace_size")
        self.ws_bytes = n.value
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        _check(load().ks_cda_create(ctypes.byref(self.cfg), self.workspace.data_ptr(), self.ws_bytes,
                                    _stream_ptr(stream), ctypes.byref(h)), "ks_cda_create")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            load().ks_cda_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int, stream=None):
        _check(load().ks_cda_step_n(self.handle, int(n), _stream_ptr(stream)), "ks_cda_step_n")

    def sync(self, timeout_ms: int = 0, stream=None) -> int:
        return int(load().ks_cda_sync(self.handle, _stream_ptr(stream), int(timeout_ms)))

    def market_slice(self, m: int) -> slice:
        return slice(m * self.A, (m + 1) * self.A)

    def read_state(self, fields=None, stream=None) -> dict:
        """Copy the state to host numpy arrays."""
        fields = list(CDA_STATE_FIELDS) if fields is None else list(fields)
        shapes = {"agent": (self.M * self.A,), "market": (self.M,), "hist": (self.M, KS_HISTORY), "one": (1,),
                  "trace": (self.trace_markets, self.trace_steps, 2)}
        v = ks_cda_state_view()
        out = {}
        for f in fields:
            dt, per = CDA_STATE_FIELDS[f]
            a = np.zeros(shapes[per], dt)
            out[f] = a
            setattr(v, f, a.ctypes.data if a.size else None)
        _check(load().ks_cda_read_state(self.handle, ctypes.byref(v), _stream_ptr(stream)), "ks_cda_read_state")
        return out
