"""The BA_DEBUG_BOUNDS build (libba_b300_debug.so, selected by BA_DEBUG_BOUNDS=1):
on valid problems no index check fails, under every solver and the adjoint, and
the checked library computes the same bits as the release one."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import dataclasses, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2510_13310_b300 import ba, scenes
out = {"lib": ba.LIB_PATH, "runs": []}
spec = dataclasses.replace(scenes.SPECS["small"], n_cams=24, n_pts=3000, seed=5)
sc = scenes.make_scene(spec)
for prec, solver in [(ba.BA_FP32, ba.BA_SOLVER_IMPLICIT), (ba.BA_FP32, ba.BA_SOLVER_EXPLICIT),
                     (ba.BA_FP32, ba.BA_SOLVER_SPARSE), (ba.BA_FP32, ba.BA_SOLVER_DENSE),
                     (ba.BA_FP64, ba.BA_SOLVER_EXPLICIT)]:
    p = ba.Problem.from_scene(sc, ba.Options(precision=prec, solver=solver))
    log = p.solve(4)
    c, q = p.get_params()
    duv, dd = p.backward(c - sc.cams_gt, q - sc.pts_gt)
    out["runs"].append({"costs": [r["cost"] for r in log], "duv": float(np.abs(duv).sum()),
                        "dd": float(np.abs(dd).sum())})
    p.close()
out["bounds"] = ba.debug_bounds(reset=True)
print(json.dumps(out))
"""


def run(debug):
    env = dict(os.environ)
    env["BA_DEBUG_BOUNDS"] = "1" if debug else "0"
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_bounds_build_clean_and_identical():
    from paper_2510_13310_b300 import build
    build.build(debug_bounds=True)
    dbg, rel = run(True), run(False)
    assert dbg["lib"].endswith("libba_b300_debug.so") and rel["lib"].endswith("libba_b300.so")
    assert dbg["bounds"] == [0, 0], dbg["bounds"]  # checks compiled in, none failed
    assert rel["bounds"] == [-1, 0]
    assert dbg["runs"] == rel["runs"]
