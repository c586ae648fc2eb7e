"""Parity of the CUDA global positioning (ba_gp_*, through the C ABI) against the
FP64 GP oracle: the pinned/free scale partition bit for bit, the FP64 cost at
an identical state, damped steps element by element, LM trajectories, and the
1M-observation scene in the configuration bench.py times for GP."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2510_13310_b300 import ba, scenes
from parity_util import check_close, kind_scale

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def gp_scene(n_cams, n_pts, lo, hi, mean, seed, **kw):
    spec = dataclasses.replace(scenes.SPECS["medium"], n_cams=n_cams, n_pts=n_pts, track_min=lo,
                               track_max=hi, track_mean=mean, seed=seed)
    return scenes.make_gp_scene(spec, **kw)


def pair(sc, **opt):
    gpu = ba.GPProblem.from_scene(sc, ba.GPOptions(**opt))
    oo = {k: v for k, v in opt.items() if k in oracle.OracleGPOptions.__dataclass_fields__}
    return gpu, oracle.OracleGP.from_scene(sc, oracle.OracleGPOptions(**oo))


def test_gp_free_partition_bit_exact():
    sc = gp_scene(15, 2000, 2, 12, 5.0, seed=3)
    depth = sc.depth.copy()
    depth[::13] = np.nan
    sc = dataclasses.replace(sc, depth=depth)
    gpu, orc = pair(sc)
    fr_g, n_g = gpu.get_free()
    fr_o, n_o = orc.free_set()
    assert n_g == n_o
    np.testing.assert_array_equal(fr_g, fr_o)
    # pinned scales report 1/d, free ones the initial value
    _, _, s = gpu.get_params()
    pin = fr_o < 0
    np.testing.assert_array_equal(s[pin], 1.0 / depth[pin])
    np.testing.assert_array_equal(s[~pin], sc.scales0[~pin])


def test_gp_cost_fp64_matches_oracle():
    sc = gp_scene(12, 3000, 2, 10, 5.0, seed=4)
    gpu, orc = pair(sc)
    F, rms = gpu.eval_cost()
    Fo, rms_o = orc.cost(sc.centres0, sc.pts0, sc.scales0)
    assert F == pytest.approx(Fo, rel=1e-12)
    assert rms == pytest.approx(rms_o, rel=1e-12)


@pytest.mark.parametrize("solver", [ba.BA_SOLVER_AUTO, ba.BA_SOLVER_DENSE])
@pytest.mark.parametrize("n_cams,n_pts,lo,hi,mean,depth_frac", [
    (12, 3000, 2, 12, 5.0, 0.5),    # several chunks per camera, ragged tracks, 11 free cameras
    (40, 6000, 3, 20, 8.0, 0.05),   # mostly free scales
    (30, 4000, 2, 8, 4.0, 1.0),     # every scale pinned
])
def test_gp_damped_step_matches_oracle(n_cams, n_pts, lo, hi, mean, depth_frac, solver):
    """Both centre-system solvers: block-Jacobi PCG on three-camera blocks (AUTO;
    11 and 29 free cameras leave a padded last block) and the tensor-core
    Cholesky-preconditioned CG."""
    spec = dataclasses.replace(scenes.SPECS["medium"], n_cams=n_cams, n_pts=n_pts, track_min=lo,
                               track_max=hi, track_mean=mean, seed=11, depth_frac=depth_frac)
    sc = scenes.make_gp_scene(spec)
    gpu, orc = pair(sc, pcg_rel_tol=1e-6, solver=solver)
    for lam in (1e-2, 1e-4):
        g = gpu.solve_damped(lam)
        o = orc.solve_step(sc.centres0, sc.pts0, sc.scales0, lam)
        assert o["status"] == 0
        # FP32 normal equations and solve: 2e-3 of each parameter kind's scale
        check_close(g["dt"], o["dt"], 2e-3, 2e-3 * kind_scale(o["dt"]), "dt")
        check_close(g["dX"], o["dX"], 2e-3, 2e-3 * kind_scale(o["dX"]), "dX")
        check_close(g["ds"], o["ds"], 2e-3, 2e-3 * np.abs(o["ds"]).max(initial=0.0), "ds")
        assert g["pred_decrease"] == pytest.approx(o["pred_decrease"], rel=1e-4)
        assert not g["dt"][sc.fixed_cams].any()
        assert not g["ds"][sc.depth > 0].any()


@pytest.mark.parametrize("solver", [ba.BA_SOLVER_AUTO, ba.BA_SOLVER_DENSE])
def test_gp_trajectory_matches_oracle(solver):
    sc = gp_scene(20, 4000, 3, 12, 6.0, seed=21)
    gpu, orc = pair(sc, solver=solver)
    log_g = gpu.solve(8)
    t_o, X_o, s_o, log_o = orc.lm(sc.centres0, sc.pts0, sc.scales0, 8)
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i
        assert a["accepted"] == b["accepted"], i
    t_g, X_g, s_g = gpu.get_params()
    print(f"GP final: centres max |dt| {np.abs(t_g - t_o).max():.3e}, points p99 "
          f"{np.percentile(np.abs(X_g - X_o).max(1), 99):.3e}")
    check_close(t_g, t_o, 0.0, 1e-4, "centres")
    assert np.percentile(np.abs(X_g - X_o).max(1), 99) < 1e-4


def test_gp_noise_free_reaches_truth():
    sc = scenes.make_gp_scene("small", noise=False, outliers=False)
    gpu = ba.GPProblem.from_scene(sc)
    log = gpu.solve(12)
    t, X, _ = gpu.get_params()
    assert log[-1]["cost"] <= 1e-9 * log[0]["cost"]
    np.testing.assert_allclose(t, sc.centres_gt, atol=2e-5)
    np.testing.assert_allclose(X, sc.pts_gt, atol=2e-5)


def test_gp_rejects_bad_input():
    sc = gp_scene(6, 200, 2, 4, 3.0, seed=5)
    bad = sc.obs_cam.copy()
    bad[0] = 99
    with pytest.raises(ba.BAError, match="invalid argument"):
        ba.GPProblem(sc.centres0, sc.pts0, bad, sc.obs_pt, sc.rays, sc.depth)
    rays = sc.rays.copy()
    rays[3, 1] = np.inf
    with pytest.raises(ba.BAError, match="invalid argument"):
        ba.GPProblem(sc.centres0, sc.pts0, sc.obs_cam, sc.obs_pt, rays, sc.depth)


def test_gp_full_size_scene_costs_match_oracle():
    """The 1M-observation geometry (200 cameras, 100k points, tracks 3-20) as a GP
    problem: three LM iterations' costs and decisions against the oracle."""
    sc = scenes.make_gp_scene("medium")
    gpu, orc = pair(sc)
    log_g = gpu.solve(3)
    _, _, _, log_o = orc.lm(sc.centres0, sc.pts0, sc.scales0, 3)
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i
        assert a["accepted"] == b["accepted"], i
    gpu.close()
