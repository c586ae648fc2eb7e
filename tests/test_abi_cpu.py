"""Host-only checks of the C-ABI library: it builds, loads and exports every symbol
include/ba_b300.h declares.  No compute call is made (no GPU here)."""
import ctypes as ct
import os
import re

import numpy as np
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


def test_debug_bounds_library_builds_and_exports_header_symbols():
    """The BA_DEBUG_BOUNDS variant exports the same symbols; the release library
    reports that it carries no index checks (site -1) without touching a device."""
    path = build.build(debug_bounds=True)
    assert path.endswith("libba_b300_debug.so")
    D = ct.CDLL(path)
    for n in _declared():
        assert hasattr(D, n), n
    assert ba.LIB_PATH.endswith("libba_b300.so") or os.environ.get("BA_DEBUG_BOUNDS") == "1"
    if not ba.LIB_PATH.endswith("_debug.so"):
        assert ba.debug_bounds() == (-1, 0)


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
    # 2^30 observations and more: refused before any array is read (32-bit kernel
    # indices plus their grid stride stay below 2^31 under the limit)
    st = L.ba_create(ct.byref(o), None, 0, None, 0, None, 1 << 30, None, None, None, None, ct.byref(h))
    assert st == ba.BA_ERR_INVALID_ARG and not h.value
    assert "sizes out of range" in L.ba_last_error().decode()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ba, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(ba, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        ba.lib()


def _noalloc_args(torch, n=5, C=3, P=4):
    return dict(cams=torch.zeros(C, 9, dtype=torch.float64), pts=torch.zeros(P, 3, dtype=torch.float64),
                obs_cam=torch.zeros(n, dtype=torch.int32), obs_pt=torch.zeros(n, dtype=torch.int32),
                obs_uv=torch.zeros(n, 2, dtype=torch.float64), depth=torch.zeros(n, dtype=torch.float64),
                out=torch.zeros(3, dtype=torch.float64), obs_mask=torch.ones(n, dtype=torch.uint8))


@pytest.mark.parametrize("change, match", [
    (lambda a, t: a.update(cams=a["cams"].float()), "cams must be"),
    (lambda a, t: a.update(pts=a["pts"].to(t.float32)), "pts must be"),
    (lambda a, t: a.update(obs_cam=a["obs_cam"].long()), "obs_cam must be"),
    (lambda a, t: a.update(obs_pt=a["obs_pt"].long()), "obs_pt must be"),
    (lambda a, t: a.update(obs_uv=a["obs_uv"].float()), "obs_uv must be"),
    (lambda a, t: a.update(depth=a["depth"].float()), "depth must be"),
    (lambda a, t: a.update(out=a["out"].float()), "out must be"),
    (lambda a, t: a.update(obs_mask=a["obs_mask"].int()), "obs_mask must be"),
    (lambda a, t: a.update(obs_uv=t.zeros(2, 5, dtype=t.float64).T), "obs_uv must be contiguous"),
    (lambda a, t: a.update(cams=t.zeros(3, 8, dtype=t.float64)), r"cams must hold"),
    (lambda a, t: a.update(pts=t.zeros(4, 2, dtype=t.float64)), r"cams must hold"),
    (lambda a, t: a.update(obs_pt=t.zeros(4, dtype=t.int32)), "need N entries"),
    (lambda a, t: a.update(depth=t.zeros(6, dtype=t.float64)), "need N entries"),
    (lambda a, t: a.update(obs_uv=t.zeros(4, 2, dtype=t.float64)), "need N entries"),
    (lambda a, t: a.update(obs_mask=t.ones(4, dtype=t.uint8)), "need N entries"),
    (lambda a, t: a.update(out=t.zeros(2, dtype=t.float64)), "out needs 3"),
    (lambda a, t: None, "one CUDA device"),  # well-formed CPU tensors: not device memory
])
def test_noalloc_binding_rejects_bad_tensors(change, match):
    """The C ABI takes bare pointers; the binding refuses what would make its kernels
    read or write out of bounds.  Every check but the device one runs on the CPU."""
    torch = pytest.importorskip("torch")
    a = _noalloc_args(torch)
    change(a, torch)
    with pytest.raises(ValueError, match=match):
        ba.eval_cost_noalloc(a["cams"], a["pts"], a["obs_cam"], a["obs_pt"], a["obs_uv"],
                             a["depth"], a["out"], obs_mask=a["obs_mask"])


def _problem_args(C=3, P=4, N=5):
    rng = np.random.default_rng(0)
    return dict(cams=np.zeros((C, 9)), pts=np.zeros((P, 3)), obs_cam=rng.integers(0, C, N).astype(np.int32),
                obs_pt=rng.integers(0, P, N).astype(np.int32), obs_uv=np.zeros((N, 2)), depth=np.zeros(N))


@pytest.mark.parametrize("change,match", [
    (lambda a: a.update(cams=np.zeros((3, 8))), r"not \[C\]\[9\]"),
    (lambda a: a.update(pts=np.zeros(10)), r"not \[P\]\[3\]"),
    (lambda a: a.update(obs_pt=np.zeros(4, np.int32)), "obs_pt: 4 elements, expected 5"),
    (lambda a: a.update(obs_uv=np.zeros((4, 2))), "observations: 8 elements, expected 10"),
    (lambda a: a.update(depth=np.zeros(6)), "depth: 6 elements, expected 5"),
])
def test_problem_binding_checks_sizes_before_the_library_reads(change, match):
    """The C ABI takes bare pointers: a short observation array would be read past
    its end, so the binding checks every size against N before ba_create."""
    a = _problem_args()
    change(a)
    with pytest.raises(ValueError, match=match):
        ba.Problem(a["cams"], a["pts"], a["obs_cam"], a["obs_pt"], a["obs_uv"], a["depth"])


def test_output_buffers_are_used_in_place_or_refused():
    """An output buffer the library writes must be the exact dtype and contiguous:
    a converted copy would receive the results instead of the caller's buffer."""
    torch = pytest.importorskip("torch")
    for bad in (np.zeros(6, np.float32), np.zeros((3, 4))[:, ::2], torch.zeros(6, dtype=torch.float32),
                torch.zeros(3, 4, dtype=torch.float64)[:, ::2]):
        with pytest.raises(ValueError, match="output"):
            ba._Arr(bad, np.float64, 6, "out", out=True)
    good = np.zeros(6)
    assert ba._Arr(good, np.float64, 6, "out", out=True).obj is good
    t = torch.zeros(6, dtype=torch.float64)
    assert ba._Arr(t, np.float64, 6, "out", out=True).ptr == t.data_ptr()
    with pytest.raises(ValueError, match="7 elements, expected 6"):
        ba._Arr(np.zeros(7), np.float64, 6, "out", out=True)
