"""Host-only checks of the C-ABI library: it builds, loads and exports every symbol
include/ba_b300.h declares.  No compute call is made (no GPU here)."""
import ctypes as ct
import os
import re

import pytest

from paper_2510_13310_b300 import ba, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ba_b300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_header_symbols():
    build.build()
    L = ba.lib()
    names = _declared()
    assert "ba_create" in names and "ba_lm_step" in names and "ba_backward" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(ba.EXPORTS)


def test_defaults_and_status_strings():
    L = ba.lib()
    o = ba._Options()
    L.ba_default_options(ct.byref(o))
    assert o.precision == ba.BA_FP32 and o.img_w == 640 and o.img_h == 480
    assert o.huber_delta == 1.0 and o.min_depth == 0.1 and o.pcg_rel_tol == 1e-6
    assert o.n_fixed == 1 and o.fixed_cams[0] == 0
    for s in range(8):
        assert L.ba_status_string(s)


def test_invalid_options_rejected_before_any_device_work():
    L = ba.lib()
    o = ba._Options()
    L.ba_default_options(ct.byref(o))
    o.pcg_rel_tol = -1.0
    h = ct.c_void_p()
    st = L.ba_create(ct.byref(o), None, 0, None, 0, None, 0, None, None, None, None, ct.byref(h))
    assert st == ba.BA_ERR_INVALID_ARG and not h.value
    o.pcg_rel_tol = 1e-6
    st = L.ba_create(ct.byref(o), None, -1, None, 0, None, 0, None, None, None, None, ct.byref(h))
    assert st == ba.BA_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ba, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(ba, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        ba.lib()
