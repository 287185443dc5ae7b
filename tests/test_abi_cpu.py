"""The C ABI library loads and exports every declared entry point; argument
validation works without a GPU (no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_2606_21784_gb300 import kineticsim as ks
from paper_2606_21784_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(ks_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = ks.load()
    declared = _declared()
    assert "ks_step_n" in declared and "ks_create_ensemble" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(ks.EXPORTS) <= declared


def test_version_and_status_strings():
    lib = ks.load()
    assert lib.ks_version() >= 0x000100
    for s in range(7):
        assert lib.ks_status_string(s)


def _cfg(**kw):
    w = wl.workload("plain_mix_8192", M=4)
    c, keep = ks.make_config(w)
    for k, v in kw.items():
        setattr(c, k, v)
    return c, keep


@pytest.mark.parametrize("field,value,status", [
    ("n_markets", 0, ks.KS_ERR_INVALID_ARG),
    ("L_all", 1, ks.KS_ERR_INVALID_ARG),
    ("L_all", 5000, ks.KS_ERR_UNSUPPORTED),
    ("A_all", 20000, ks.KS_ERR_UNSUPPORTED),
    ("A_all", -1, ks.KS_ERR_INVALID_ARG),
    ("zi_qmax", 0, ks.KS_ERR_INVALID_ARG),
    ("zi_qmax", 300, ks.KS_ERR_UNSUPPORTED),
    ("mom_lookback", 9, ks.KS_ERR_INVALID_ARG),
    ("tie_rule", 7, ks.KS_ERR_INVALID_ARG),
    ("trace_markets", 5, ks.KS_ERR_INVALID_ARG),
])
def test_validation_errors(field, value, status):
    c, keep = _cfg(**{field: value})
    n = ctypes.c_size_t(0)
    rc = ks.load().ks_workspace_size(ctypes.byref(c), ctypes.byref(n))
    assert rc == status
    assert ks.load().ks_last_error()


def test_mix_must_sum_to_100():
    c, keep = _cfg()
    c.mix_pct[0] = 50
    with pytest.raises(ks.KsError) as e:
        ks.ks_workspace_size(c)
    assert e.value.status == ks.KS_ERR_INVALID_ARG


def test_workspace_size_matches_layout():
    w = wl.workload("plain_mix_8192")
    c, keep = ks.make_config(w)
    n = ks.ks_workspace_size(c)
    N = w["M"] * w["A"]
    assert 16 * N <= n <= 16 * N + 16 * w["M"] * 8 + 4096


def test_create_rejects_small_or_misaligned_workspace():
    c, keep = _cfg()
    lib = ks.load()
    h = ctypes.c_void_p(0)
    need = ks.ks_workspace_size(c)
    assert lib.ks_create_ensemble(ctypes.byref(c), 256, need - 1, None, ctypes.byref(h)) == ks.KS_ERR_WORKSPACE_TOO_SMALL
    assert lib.ks_create_ensemble(ctypes.byref(c), 257, need, None, ctypes.byref(h)) == ks.KS_ERR_INVALID_ARG
    assert lib.ks_create_ensemble(ctypes.byref(c), None, need, None, ctypes.byref(h)) == ks.KS_ERR_INVALID_ARG
    assert h.value is None


def test_null_handles_are_rejected():
    lib = ks.load()
    assert lib.ks_step_n(None, 1, None) == ks.KS_ERR_INVALID_ARG
    assert lib.ks_sync(None, None, 0) == ks.KS_ERR_INVALID_ARG
    assert lib.ks_read_state(None, None, None) == ks.KS_ERR_INVALID_ARG


# --------------------------------------------------------------------------
# the paper-agent ensemble (ks_paper_*)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("field,value,status", [
    ("n_markets", 0, ks.KS_ERR_INVALID_ARG),
    ("L", 1, ks.KS_ERR_UNSUPPORTED),
    ("L", 5000, ks.KS_ERR_UNSUPPORTED),
    ("A", -1, ks.KS_ERR_UNSUPPORTED),
    ("A", 20000, ks.KS_ERR_UNSUPPORTED),
    ("qmax", 0, ks.KS_ERR_INVALID_ARG),
    ("qmax", 256, ks.KS_ERR_INVALID_ARG),
    ("noise_halfwidth", -1, ks.KS_ERR_INVALID_ARG),
    ("maker_half_spread", 200, ks.KS_ERR_INVALID_ARG),
    ("mom_pct", 90, ks.KS_ERR_INVALID_ARG),
    ("tie_rule", 3, ks.KS_ERR_INVALID_ARG),
])
def test_paper_validation_errors(field, value, status):
    c = ks.make_paper_config(wl.workload("paper_8192_256", M=4))
    setattr(c, field, value)
    n = ctypes.c_size_t(0)
    assert ks.load().ks_paper_workspace_size(ctypes.byref(c), ctypes.byref(n)) == status
    assert ks.load().ks_last_error()


def test_paper_workspace_and_create_checks():
    lib = ks.load()
    w = wl.workload("paper_8192_1024")
    c = ks.make_paper_config(w, trace_markets=2, trace_steps=10)
    n = ctypes.c_size_t(0)
    assert lib.ks_paper_workspace_size(ctypes.byref(c), ctypes.byref(n)) == ks.KS_OK
    ML = w["M"] * w["L"]
    assert 8 * ML <= n.value <= 8 * ML + 64 * w["M"] + 4096  # bid + ask books, 64 B of scalars, trace
    h = ctypes.c_void_p(0)
    assert lib.ks_paper_create(ctypes.byref(c), 256, n.value - 1, None, ctypes.byref(h)) == \
        ks.KS_ERR_WORKSPACE_TOO_SMALL
    assert lib.ks_paper_create(ctypes.byref(c), 257, n.value, None, ctypes.byref(h)) == ks.KS_ERR_INVALID_ARG
    assert h.value is None
    assert lib.ks_paper_step_n(None, 1, None) == ks.KS_ERR_INVALID_ARG
    assert lib.ks_paper_sync(None, None, 0) == ks.KS_ERR_INVALID_ARG
