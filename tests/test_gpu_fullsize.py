"""Parity at the workloads' full sizes, in the configuration bench.py times.

The 1M-observation scene (200 cameras, 100k points, FP32, automatic solver):
per-iteration costs of a short LM run against the oracle's, and the normal
equation blocks at an identical state (camera and point blocks in full, W on a
sample of observations).  The 8M-observation extraction scene (1,500 cameras,
1M points, thresholds (15, 2), 4 px residual drop at every 5th iteration): the
active sets and compaction maps bit for bit against the oracle's extraction of
the same state."""
import numpy as np
import pytest

import oracle
from paper_2510_13310_b300 import ba, scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def medium():
    return scenes.make_scene("medium")


def test_bench_workload_blocks_at_identical_state(medium):
    sc = medium
    gpu = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP32))
    lin = gpu.linearize(want_W=True)
    act = gpu.get_active()
    orc = oracle.OracleBA.from_scene(sc)
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    for key in ("cam_mask", "pt_mask", "obs_mask", "cam_rank", "pt_rank"):
        np.testing.assert_array_equal(act[key], ext[key], err_msg=key)
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    live = ext["cam_mask"].astype(bool)
    # FP32 sums of ~5,000 observations per camera, ~10 per point
    assert rel_err(lin["U"][live], ne["U"][live]) < 1e-3
    assert rel_err(lin["gc"][live], ne["gc"][live]) < 1e-3
    assert rel_err(lin["V"], ne["V"]) < 2e-4
    assert rel_err(lin["gp"], ne["gp"]) < 2e-4
    idx = np.random.default_rng(0).choice(sc.n_obs, 20000, replace=False)
    assert rel_err(lin["W"][idx], ne["W"][idx]) < 2e-4
    gpu.close()


def test_bench_workload_lm_costs_match_oracle(medium):
    sc = medium
    gpu = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP32))
    log_g = gpu.solve(3)
    orc = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(solver=1))
    _, _, log_o = orc.lm(sc.cams0, sc.pts0, 3)
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i
        assert a["accepted"] == b["accepted"], i
        assert a["n_obs_act"] == b["n_obs_act"], i
    gpu.close()


def test_large_extraction_workload_bit_exact():
    sc = scenes.make_scene("large")
    opt = dict(min_cam_obs=15, min_pt_obs=2, drop_residual_px=4.0)
    # converge first (no automatic drop), then the 4 px drop and the (15, 2)
    # thresholds at that state, on both sides
    gpu = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP32, extract_every=0, **opt))
    log = gpu.solve(15)
    cams, pts = gpu.get_params()
    gpu.extract(drop=True)
    g = gpu.get_active()
    orc = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(**opt))
    geom, res = orc.predicate(cams, pts)
    alive = ~((geom == 1) & (res > 4.0))
    e = orc.extract((geom.astype(bool) & alive).astype(np.uint8))
    for key in ("cam_mask", "pt_mask", "obs_mask", "cam_rank", "pt_rank"):
        np.testing.assert_array_equal(g[key], e[key], err_msg=key)
    om = g["obs_mask"].astype(bool)
    print(f"rmse {log[-1]['rmse_px']:.3f} px; kept: outliers {om[sc.is_outlier].mean():.4f}, "
          f"inliers {om[~sc.is_outlier].mean():.4f}; cameras {g['cam_mask'].mean():.4f}, "
          f"points {g['pt_mask'].mean():.4f}")
    # a non-degenerate active set: the outliers go, most inliers stay
    assert (~om[sc.is_outlier]).mean() > 0.9
    assert om[~sc.is_outlier].mean() > 0.5
    gpu.close()
