"""ctypes front-end of the C oracle in ``ks_oracle.c`` (test infrastructure).

The oracle is a plain single-threaded CPU simulator written from the paper
(Sec. II-A Eq. 1-2 clearing, Sec. III-D tie rule, Sec. IV-C allocation) and
from the stated readings of the benchmark configurations.  It shares no code
with the CUDA library; the only thing both sides receive in common is the
seeded workload description (ensemble sizes and agent parameters).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may use it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libks_oracle.so")
_lock = threading.Lock()
_lib = None

HIST = 9
ZI, MOM, MR = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ks_oracle.c into a shared library with gcc (no GPU code)."""
    os.makedirs(_BUILD, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("carry_book", ctypes.c_int32),
        ("cancel_thresh", ctypes.c_uint32),
        ("mix_pct", ctypes.c_int32 * 3),
        ("zi_offset", ctypes.c_int32),
        ("zi_qmax", ctypes.c_int32),
        ("mom_lookback", ctypes.c_int32),
        ("mom_offset_max", ctypes.c_int32),
        ("mr_offset_max", ctypes.c_int32),
        ("rb_qmax", ctypes.c_int32),
        ("mlp_pct", ctypes.c_int32),
        ("tie_rule", ctypes.c_int32),
    ]


class MarketScalars(ctypes.Structure):
    _fields_ = [
        ("last", ctypes.c_int32),
        ("hist", ctypes.c_int32 * HIST),
        ("fund", ctypes.c_int32),
        ("trades", ctypes.c_int32),
        ("last_v", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("sum_p", ctypes.c_int64),
        ("sum_v", ctypes.c_int64),
        ("hash", ctypes.c_uint64),
    ]


class _Agents(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("qty", "side", "tick", "atype", "mlp", "inv", "cash")]


class _Replay(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("side", "tick", "qty")]


class _Options(ctypes.Structure):
    _fields_ = [("mlp_w", ctypes.c_void_p), ("rec_agents", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("rec_out", ctypes.c_void_p), ("rec_cap", ctypes.c_int64), ("rec_count", ctypes.c_int64),
                ("mlp_checked", ctypes.c_int64), ("mlp_mismatch", ctypes.c_int64), ("logit_out", ctypes.c_void_p)]


MLP_IN, MLP_H, MLP_OUT, N_RAW, REC_WORDS = 32, 64, 37, 18, 22


class PaperParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("noise_halfwidth", ctypes.c_int32), ("p_mkt_q32", ctypes.c_uint32),
                ("qmax", ctypes.c_int32), ("maker_half_spread", ctypes.c_int32), ("mom_pct", ctypes.c_int32),
                ("maker_pct", ctypes.c_int32), ("tie_rule", ctypes.c_int32), ("window", ctypes.c_int32)]


class PaperMarket(ctypes.Structure):
    _fields_ = [("last", ctypes.c_int32), ("mid2", ctypes.c_int32), ("trades", ctypes.c_int32),
                ("last_v", ctypes.c_int32), ("sum_p", ctypes.c_int64), ("sum_v", ctypes.c_int64),
                ("hash", ctypes.c_uint64), ("base", ctypes.c_int64)]


PAPER_NOISE, PAPER_MOMENTUM, PAPER_MAKER = 0, 1, 2


class _ClearResult(ctypes.Structure):
    _fields_ = [
        ("vstar", ctypes.c_int64),
        ("pstar", ctypes.c_int32),
        ("p_buy", ctypes.c_int32),
        ("p_sell", ctypes.c_int32),
        ("argmax", ctypes.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # KS_ORACLE_LIB lets the mutation tests load a deliberately broken copy
            lib = ctypes.CDLL(os.environ.get("KS_ORACLE_LIB") or build())
            P = ctypes.POINTER
            lib.ko_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            lib.ko_philox4x32_10.restype = None
            lib.ko_trace_hash_update.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32]
            lib.ko_trace_hash_update.restype = ctypes.c_uint64
            lib.ko_clear_book.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, P(_ClearResult)]
            lib.ko_clear_book.restype = ctypes.c_int
            lib.ko_allocate.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
            lib.ko_allocate.restype = ctypes.c_int
            lib.ko_init_market.argtypes = [P(Params), ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32,
                                           P(_Agents), P(MarketScalars)]
            lib.ko_init_market.restype = ctypes.c_int
            lib.ko_run_market.argtypes = [P(Params), ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32,
                                          P(_Agents), P(MarketScalars), ctypes.c_uint32, ctypes.c_uint32,
                                          P(_Replay), ctypes.c_void_p, ctypes.c_void_p, P(_Options)]
            lib.ko_run_market.restype = ctypes.c_int
            lib.ko_mlp_nparam.argtypes = []
            lib.ko_mlp_nparam.restype = ctypes.c_int32
            lib.ko_mlp_forward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
            lib.ko_mlp_forward.restype = ctypes.c_int
            lib.ko_mlp_loss_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int64, P(ctypes.c_double), ctypes.c_void_p]
            lib.ko_mlp_loss_grad.restype = ctypes.c_int
            lib.ko_mlp_features.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
            lib.ko_mlp_features.restype = None
            lib.ko_mlp_action.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int32),
                                          P(ctypes.c_int32), P(ctypes.c_int32)]
            lib.ko_mlp_action.restype = None
            lib.ko_adam_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double]
            lib.ko_adam_step.restype = None
            lib.ko_splitmix64_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
            lib.ko_splitmix64_draw.restype = ctypes.c_uint64
            lib.ko_paper_class.argtypes = [P(PaperParams), ctypes.c_uint64]
            lib.ko_paper_class.restype = ctypes.c_int32
            lib.ko_paper_order.argtypes = [P(PaperParams), ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32,
                                           ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)]
            lib.ko_paper_order.restype = None
            lib.ko_paper_init.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, P(PaperMarket)]
            lib.ko_paper_init.restype = ctypes.c_int
            lib.ko_paper_run.argtypes = [P(PaperParams), ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p, P(PaperMarket), ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_void_p]
            lib.ko_paper_run.restype = ctypes.c_int
            lib.ko_cda_run.argtypes = [P(Params), ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32, P(_Agents),
                                       ctypes.c_void_p, P(MarketScalars), ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       P(ctypes.c_int64), P(_Replay)]
            lib.ko_cda_run.restype = ctypes.c_int
            lib.ko_rule_decision.argtypes = [P(Params), ctypes.c_int32, ctypes.c_int32, P(MarketScalars),
                                             P(ctypes.c_uint32), P(ctypes.c_int32)]
            lib.ko_rule_decision.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# ---------------------------------------------------------------------------
# RNG and hash
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block (Salmon et al., SC'11) for a 4-word counter and 2-word key."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.ko_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def trace_hash_update(h: int, step: int, pstar: int, vol: int) -> int:
    return int(_load().ko_trace_hash_update(h, step, pstar, vol))


# ---------------------------------------------------------------------------
# Clearing of one book and greedy allocation
# ---------------------------------------------------------------------------
@dataclass
class Clearing:
    dcum: np.ndarray
    scum: np.ndarray
    vol: np.ndarray
    vstar: int
    pstar: int
    p_buy: int
    p_sell: int
    argmax: int


def clear_book(buy, sell, tie_rule: int = 0) -> Clearing:
    """Uniform-price call-auction clearing of one aggregated book (Sec. II-A, Eq. 1-2)."""
    buy = np.ascontiguousarray(buy, dtype=np.int64)
    sell = np.ascontiguousarray(sell, dtype=np.int64)
    L = buy.shape[0]
    assert sell.shape[0] == L
    d = np.zeros(L, np.int64)
    s = np.zeros(L, np.int64)
    v = np.zeros(L, np.int64)
    r = _ClearResult()
    rc = _load().ko_clear_book(L, _ptr(buy), _ptr(sell), tie_rule, _ptr(d), _ptr(s), _ptr(v), ctypes.byref(r))
    if rc != 0:
        raise ValueError(f"ko_clear_book failed: {rc}")
    return Clearing(d, s, v, int(r.vstar), int(r.pstar), int(r.p_buy), int(r.p_sell), int(r.argmax))


def allocate(L: int, side, tick, qty, vstar: int) -> np.ndarray:
    """Greedy price-then-agent-index allocation of V* (Sec. IV-C)."""
    side = np.ascontiguousarray(side, dtype=np.int32)
    tick = np.ascontiguousarray(tick, dtype=np.int32)
    qty = np.ascontiguousarray(qty, dtype=np.int32)
    A = side.shape[0]
    fill = np.zeros(A, np.int32)
    rc = _load().ko_allocate(L, A, _ptr(side), _ptr(tick), _ptr(qty), int(vstar), _ptr(fill))
    if rc != 0:
        raise ValueError(f"ko_allocate failed: {rc}")
    return fill


# ---------------------------------------------------------------------------
# Market simulation
# ---------------------------------------------------------------------------
@dataclass
class Market:
    """Full state of one market as the oracle holds it."""
    m: int
    L: int
    A: int
    qty: np.ndarray
    side: np.ndarray
    tick: np.ndarray
    atype: np.ndarray
    mlp: np.ndarray
    inv: np.ndarray
    cash: np.ndarray
    sc: MarketScalars = field(default_factory=MarketScalars)

    def _agents(self) -> _Agents:
        return _Agents(*[_ptr(getattr(self, n)) for n in ("qty", "side", "tick", "atype", "mlp", "inv", "cash")])

    @property
    def last(self) -> int:
        return int(self.sc.last)

    @property
    def hist(self) -> np.ndarray:
        return np.array(list(self.sc.hist), dtype=np.int32)

    def scalars(self) -> dict:
        sc = self.sc
        return dict(last=int(sc.last), hist=list(sc.hist), fund=int(sc.fund), trades=int(sc.trades),
                    last_v=int(sc.last_v), sum_p=int(sc.sum_p), sum_v=int(sc.sum_v), hash=int(sc.hash))


def make_params(p: dict) -> Params:
    """Build the oracle's parameter block from a workload description dict."""
    P = Params()
    P.seed = int(p["seed"])
    P.carry_book = int(p["carry_book"])
    P.cancel_thresh = int(p["cancel_thresh_q32"])
    for i in range(3):
        P.mix_pct[i] = int(p["mix_pct"][i])
    P.zi_offset = int(p["zi_offset"])
    P.zi_qmax = int(p["zi_qmax"])
    P.mom_lookback = int(p["mom_lookback"])
    P.mom_offset_max = int(p["mom_offset_max"])
    P.mr_offset_max = int(p["mr_offset_max"])
    P.rb_qmax = int(p["rb_qmax"])
    P.mlp_pct = int(p.get("mlp_pct", 0))
    P.tie_rule = int(p.get("tie_rule", 0))
    return P


def init_market(params: dict, m: int, L: int, A: int) -> Market:
    z = lambda dt: np.zeros(max(A, 1), dt)[:A]  # noqa: E731
    mk = Market(m, L, A, z(np.int32), z(np.int32), z(np.int32), z(np.int32), z(np.int32), z(np.int32), z(np.int64))
    P = make_params(params)
    rc = _load().ko_init_market(ctypes.byref(P), m, L, A, ctypes.byref(mk._agents()), ctypes.byref(mk.sc))
    if rc != 0:
        raise ValueError(f"ko_init_market failed: {rc}")
    return mk


def run_market(params: dict, mk: Market, s0: int, n: int, replay=None, want_trace: bool = True, mlp_w=None,
               rec_agents: int = 0, rec_cap: int = 0, stats: dict | None = None, want_logits: bool = False):
    """Advance ``mk`` in place over steps [s0, s0+n).  Returns (trace_p, trace_v) or None.

    ``replay``: optional dict of int32 arrays ``side``, ``tick``, ``qty`` of shape (n, A)
    holding the decisions of MLP agents (side 2 = pass).  ``mlp_w``: fp64 policy
    parameters (MLP agents decide with them, or are checked against them when
    replaying).  ``rec_agents`` / ``rec_cap``: record rule decisions of agents
    a < rec_agents.  ``stats`` (optional dict) receives ``records`` (int32
    [count, 22]), ``mlp_checked`` and ``mlp_mismatch``, and with
    ``want_logits`` (needs ``mlp_w``) ``logits``: fp64 [n, A, 37] of every
    policy decision, NaN where no policy decision was taken.
    """
    P = make_params(params)
    tp = np.zeros(max(n, 1), np.int32)
    tv = np.zeros(max(n, 1), np.int32)
    rp = None
    keep = []
    if replay is not None:
        arrs = [np.ascontiguousarray(replay[k], dtype=np.int32) for k in ("side", "tick", "qty")]
        for a in arrs:
            assert a.size == n * mk.A
        keep = arrs
        rp = ctypes.byref(_Replay(*[_ptr(a) for a in arrs]))
    opt = _Options()
    if mlp_w is not None:
        w = np.ascontiguousarray(mlp_w, dtype=np.float64)
        assert w.size == mlp_nparam()
        keep.append(w)
        opt.mlp_w = _ptr(w)
    logits = None
    if want_logits:
        assert mlp_w is not None
        logits = np.full((max(n, 1), max(mk.A, 1), MLP_OUT), np.nan, np.float64)
        opt.logit_out = _ptr(logits)
    rec = None
    if rec_agents > 0 and rec_cap > 0:
        rec = np.zeros((rec_cap, REC_WORDS), np.int32)
        opt.rec_agents = rec_agents
        opt.rec_out = _ptr(rec)
        opt.rec_cap = rec_cap
    rc = _load().ko_run_market(ctypes.byref(P), mk.m, mk.L, mk.A, ctypes.byref(mk._agents()), ctypes.byref(mk.sc),
                               s0, n, rp, _ptr(tp) if want_trace else None, _ptr(tv) if want_trace else None,
                               ctypes.byref(opt))
    del keep
    if rc != 0:
        raise ValueError(f"ko_run_market failed: {rc}")
    if stats is not None:
        stats["records"] = rec[: opt.rec_count] if rec is not None else np.zeros((0, REC_WORDS), np.int32)
        stats["mlp_checked"] = int(opt.mlp_checked)
        stats["mlp_mismatch"] = int(opt.mlp_mismatch)
        if logits is not None:
            stats["logits"] = logits[:n, :mk.A]
    return (tp[:n], tv[:n]) if want_trace else None


# ---------------------------------------------------------------------------
# MLP policy (fp64)
# ---------------------------------------------------------------------------
def mlp_nparam() -> int:
    return int(_load().ko_mlp_nparam())


def mlp_pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    """fp64 parameter vector: W1[64,32], b1, W2[64,64], b2, W3[37,64], b3."""
    return np.concatenate([np.asarray(a, np.float64).ravel() for a in (W1, b1, W2, b2, W3, b3)])


def mlp_unpack(w):
    w = np.asarray(w, np.float64)
    shapes = [(MLP_H, MLP_IN), (MLP_H,), (MLP_H, MLP_H), (MLP_H,), (MLP_OUT, MLP_H), (MLP_OUT,)]
    out, i = [], 0
    for sh in shapes:
        k = int(np.prod(sh))
        out.append(w[i:i + k].reshape(sh))
        i += k
    return out


def mlp_forward(w, X) -> np.ndarray:
    """Logits [n, 37] of feature rows X [n, 32] (fp64)."""
    w = np.ascontiguousarray(w, np.float64)
    X = np.ascontiguousarray(X, np.float64)
    Z = np.zeros((X.shape[0], MLP_OUT), np.float64)
    _load().ko_mlp_forward(_ptr(w), _ptr(X), X.shape[0], _ptr(Z))
    return Z


def mlp_loss_grad(w, X, side, offset, logq):
    """Mean behaviour-cloning loss and its gradient (fp64)."""
    w = np.ascontiguousarray(w, np.float64)
    X = np.ascontiguousarray(X, np.float64)
    side = np.ascontiguousarray(side, np.int32)
    offset = np.ascontiguousarray(offset, np.int32)
    logq = np.ascontiguousarray(logq, np.float64)
    g = np.zeros(mlp_nparam(), np.float64)
    loss = ctypes.c_double(0)
    rc = _load().ko_mlp_loss_grad(_ptr(w), _ptr(X), _ptr(side), _ptr(offset), _ptr(logq), X.shape[0],
                                  ctypes.byref(loss), _ptr(g))
    if rc != 0:
        raise ValueError(rc)
    return float(loss.value), g


def adam_step(w, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One fp64 Adam step in place on w, m, v."""
    for a in (w, g, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    _load().ko_adam_step(_ptr(w), _ptr(g), _ptr(m), _ptr(v), w.size, int(t), lr, b1, b2, eps)


def mlp_features(raw, A: int) -> np.ndarray:
    raw = np.ascontiguousarray(raw, np.int32)
    x = np.zeros(MLP_IN, np.float64)
    _load().ko_mlp_features(_ptr(raw), int(A), _ptr(x))
    return x


def mlp_action(z, words, qmax: int):
    z = np.ascontiguousarray(z, np.float64)
    w = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in words])
    sd, oi, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _load().ko_mlp_action(_ptr(z), w, int(qmax), ctypes.byref(sd), ctypes.byref(oi), ctypes.byref(q))
    return int(sd.value), int(oi.value), int(q.value)


def simulate(params: dict, m: int, L: int, A: int, steps: int, replay=None, mlp_w=None):
    """Initialise market m and run ``steps`` steps from step 0; returns (market, trace_p, trace_v)."""
    mk = init_market(params, m, L, A)
    tp, tv = run_market(params, mk, 0, steps, replay=replay, mlp_w=mlp_w)
    return mk, tp, tv


# ---------------------------------------------------------------------------
# The paper's own agents on a tick-aggregated book (Sec. III-C, III-G)
# ---------------------------------------------------------------------------
def make_paper_params(p: dict) -> PaperParams:
    return PaperParams(int(p["seed"]) & 0xFFFFFFFFFFFFFFFF, int(p["noise_halfwidth"]), int(p["p_mkt_q32"]),
                       int(p["qmax"]), int(p["maker_half_spread"]), int(p["mom_pct"]), int(p["maker_pct"]),
                       int(p.get("tie_rule", 0)), int(p.get("window", 0)))


def splitmix64_draw(seed: int, gid: int, step: int, channel: int) -> int:
    """Output number gid*2^35 + 8*step + channel of SplitMix64 with state ``seed``."""
    return int(_load().ko_splitmix64_draw(seed & 0xFFFFFFFFFFFFFFFF, gid & 0xFFFFFFFFFFFFFFFF, step, channel))


def paper_class(params: dict, gid: int) -> int:
    P = make_paper_params(params)
    return int(_load().ko_paper_class(ctypes.byref(P), gid))


def paper_order(params: dict, L: int, gid: int, a: int, s: int, cls: int, mid2: int, ret: int):
    """(side, tick, qty) of one agent's order at step s (side 0 buy, 1 sell)."""
    P = make_paper_params(params)
    sd, tk, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _load().ko_paper_order(ctypes.byref(P), L, gid, a, s, cls, mid2, ret, ctypes.byref(sd), ctypes.byref(tk),
                           ctypes.byref(q))
    return int(sd.value), int(tk.value), int(q.value)


@dataclass
class PaperBook:
    market: int
    L: int
    A: int
    bid: np.ndarray
    ask: np.ndarray
    sc: PaperMarket = field(default_factory=PaperMarket)

    def scalars(self) -> dict:
        return {k: int(getattr(self.sc, k))
                for k in ("last", "mid2", "trades", "last_v", "sum_p", "sum_v", "hash", "base")}


def paper_init(market: int, L: int, A: int) -> PaperBook:
    bk = PaperBook(market, L, A, np.zeros(L, np.int32), np.zeros(L, np.int32))
    if _load().ko_paper_init(L, _ptr(bk.bid), _ptr(bk.ask), ctypes.byref(bk.sc)) != 0:
        raise ValueError("ko_paper_init failed")
    return bk


def paper_run(params: dict, bk: PaperBook, s0: int, n: int, want_trace: bool = True):
    """Advance ``bk`` in place over steps [s0, s0+n); returns (trace_p, trace_v) or None."""
    P = make_paper_params(params)
    tr = np.zeros((max(n, 1), 2), np.int32)
    rc = _load().ko_paper_run(ctypes.byref(P), bk.market, bk.L, bk.A, _ptr(bk.bid), _ptr(bk.ask),
                              ctypes.byref(bk.sc), s0, n, _ptr(tr) if want_trace else None)
    if rc != 0:
        raise ValueError(f"ko_paper_run failed: {rc}")
    return (tr[:n, 0].copy(), tr[:n, 1].copy()) if want_trace else None


def paper_simulate(params: dict, market: int, L: int, A: int, steps: int):
    bk = paper_init(market, L, A)
    tp, tv = paper_run(params, bk, 0, steps)
    return bk, tp, tv


# ---------------------------------------------------------------------------
# Continuous double auction (the main model's agents, continuous matching)
# ---------------------------------------------------------------------------
def cda_init(params: dict, m: int, L: int, A: int):
    """A CDA market: the main model's initial state plus arrival stamps (-1: no resting order)."""
    mk = init_market(params, m, L, A)
    mk.stamp = np.full(max(A, 1), -1, np.int64)[:A]
    return mk


def cda_run(params: dict, mk: Market, s0: int, n: int, fills_cap: int = 0, inject=None):
    """Advance CDA market ``mk`` over steps [s0, s0+n); returns (trace_p, trace_v, fills)
    with fills an int32 [count, 5] log (step, incoming agent, resting agent, tick, qty)
    when ``fills_cap`` > 0.  ``inject`` (tests): dict of int32 arrays ``side``, ``tick``,
    ``qty`` of shape (n, A) replacing the decisions of deciding agents."""
    P = make_params(params)
    keep = []
    inj = None
    if inject is not None:
        keep = [np.ascontiguousarray(inject[k], dtype=np.int32) for k in ("side", "tick", "qty")]
        for a in keep:
            assert a.size == n * mk.A
        inj = ctypes.byref(_Replay(*[_ptr(a) for a in keep]))
    tp = np.zeros(max(n, 1), np.int32)
    tv = np.zeros(max(n, 1), np.int32)
    fl = np.zeros((max(fills_cap, 1), 5), np.int32)
    cnt = ctypes.c_int64(0)
    rc = _load().ko_cda_run(ctypes.byref(P), mk.m, mk.L, mk.A, ctypes.byref(mk._agents()), _ptr(mk.stamp),
                            ctypes.byref(mk.sc), s0, n, _ptr(tp), _ptr(tv), _ptr(fl) if fills_cap > 0 else None,
                            int(fills_cap), ctypes.byref(cnt), inj)
    del keep
    if rc != 0:
        raise ValueError(f"ko_cda_run failed: {rc}")
    return tp[:n], tv[:n], fl[:min(int(cnt.value), fills_cap)]


def cda_next(mk: Market) -> np.ndarray:
    """Time-priority successor of every resting order: the agent resting next at
    the same side and tick (by arrival stamp), -1 for the last one and for agents
    without a resting order."""
    nxt = np.full(mk.A, -1, np.int32)
    live = np.nonzero(mk.qty > 0)[0]
    keys = {}
    for a in live:
        keys.setdefault((int(mk.side[a]), int(mk.tick[a])), []).append(int(a))
    for ags in keys.values():
        ags.sort(key=lambda x: int(mk.stamp[x]))
        for x, y in zip(ags, ags[1:]):
            nxt[x] = y
    return nxt


def rule_decision(params: dict, L: int, atype: int, last: int, hist, fund: int, words):
    """(side, tick, qty) of a rule agent of class ``atype`` with draw words ``words``
    in a market whose last clearing tick, history (newest first) and fundamental
    are given."""
    P = make_params(params)
    ms = MarketScalars()
    ms.last = int(last)
    for j in range(HIST):
        ms.hist[j] = int(hist[j])
    ms.fund = int(fund)
    w = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in words])
    out = (ctypes.c_int32 * 3)()
    _load().ko_rule_decision(ctypes.byref(P), int(L), int(atype), ctypes.byref(ms), w, out)
    return int(out[0]), int(out[1]), int(out[2])
