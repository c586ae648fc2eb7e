"""Host-side observation layout of ba_create (csrc/layout.cu), on the CPU.

Builds tests/layout_check.cu with the layout builder (host code only, no device
code) and runs it: the point-order and camera-order permutations, offsets,
tiles, metadata offsets, camera chunks and co-visibility runs are compared with
brute-force definitions on random scenes (long and short tracks, empty points
and cameras, no observations); duplicate observations, out-of-range indices,
non-finite values and over-long tracks are rejected; and the layout is
bit-identical for 1, 3 and 7 host threads and for the wide-key sort path."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.mark.skipif(not (os.path.exists(NVCC) or shutil.which("nvcc")), reason="needs nvcc")
def test_layout_invariants_errors_and_thread_independence(tmp_path):
    exe = tmp_path / "layout_check"
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                           "--expt-relaxed-constexpr", "-Wno-deprecated-declarations", "-o", str(exe),
                           os.path.join(ROOT, "tests", "layout_check.cu"),
                           os.path.join(ROOT, "paper_2510_13310_b300", "csrc", "layout.cu"), "-lpthread"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stderr[-4000:]
