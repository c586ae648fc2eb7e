"""Parity at the workloads' full sizes, in the configuration bench.py times.

The 1M-observation scene (200 cameras, 100k points, FP32, automatic solver): the
normal-equation blocks at an identical state element by element (W on a sample),
and the configured run of 30 LM iterations against the oracle's, with the final
pose and point differences stated.  The 8M-observation scene (1,500 cameras, 1M
points) under its configured schedule: 4 px residual drop at iterations 5 and
10 with thresholds (15, 2), masks and compaction maps bit for bit at every
extraction, the trajectory segment by segment against the oracle."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2510_13310_b300 import ba, scenes
from parity_util import check_blocks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


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
    idx = np.random.default_rng(0).choice(sc.n_obs, 20000, replace=False)
    # FP32 sums of ~5,000 observations per camera and ~10 per point
    print(check_blocks(lin, ne, orc, sc.cams0, sc.pts0, ext["obs_mask"], live, 1e-4, W_rows=idx))
    gpu.close()


def pose_diff(c1, c2):
    rot = np.degrees(np.linalg.norm((Rotation.from_rotvec(c1[:, :3]) *
                                     Rotation.from_rotvec(c2[:, :3]).inv()).as_rotvec(), axis=1))
    return dict(rot_deg=rot.max(), t=np.abs(c1[:, 3:6] - c2[:, 3:6]).max(),
                f_px=np.abs(c1[:, 6] - c2[:, 6]).max(), k=np.abs(c1[:, 7:9] - c2[:, 7:9]).max())


def test_bench_workload_30_iterations_match_oracle(medium):
    """The configured 1M-observation run: 30 LM iterations of the FP32 path against
    the FP64 oracle (CG with the same stopping rule).  Costs within 1e-5 at every
    iteration and the same accept decisions; final differences stated per camera
    parameter kind and, for points, over the well-determined ones (the oracle's
    final error against the truth below 1: about 90 points of 100k with tracks of
    3-4 containing outliers drift far on both sides and are counted separately)."""
    sc = medium
    gpu = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP32))
    log_g = gpu.solve(30)
    cg, pg = gpu.get_params()
    gpu.close()
    orc = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(solver=1))
    co, po, log_o = orc.lm(sc.cams0, sc.pts0, 30)
    rel = [a["cost"] / b["cost"] - 1 for a, b in zip(log_g, log_o)]
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i
        assert a["accepted"] == b["accepted"], i
        assert a["n_obs_act"] == b["n_obs_act"], i
    good = np.linalg.norm(po - sc.pts_gt, axis=1) < 1.0
    dp = np.linalg.norm(pg - po, axis=1)
    d = pose_diff(cg, co)
    pct = np.percentile(dp[good], [50, 99, 100])
    print(f"30 iterations: max |cost rel| {np.abs(rel).max():.2e}; GPU - oracle final: rotation "
          f"{d['rot_deg']:.2e} deg, translation {d['t']:.2e}, focal {d['f_px']:.2e} px, k {d['k']:.2e}; "
          f"points (well determined: {good.sum()} of {good.size}) |dp| median {pct[0]:.2e}, "
          f"p99 {pct[1]:.2e}, max {pct[2]:.2e}; final RMSE {log_g[-1]['rmse_px']:.6f} vs "
          f"{log_o[-1]['rmse_px']:.6f} px")
    gt_g, gt_o = pose_diff(cg, sc.cams_gt), pose_diff(co, sc.cams_gt)
    print(f"against the truth: GPU rotation {gt_g['rot_deg']:.4f} deg, oracle {gt_o['rot_deg']:.4f} deg; "
          f"point error median GPU {np.median(np.linalg.norm(pg - sc.pts_gt, axis=1)[good]):.3e}, "
          f"oracle {np.median(np.linalg.norm(po - sc.pts_gt, axis=1)[good]):.3e}")
    assert good.sum() >= 0.998 * good.size
    assert d["rot_deg"] < 1e-2 and d["t"] < 2e-3 and d["f_px"] < 1.0
    assert pct[0] < 1e-4 and pct[1] < 1e-2


def test_large_workload_configured_schedule():
    """configs' 8M-observation run as specified: thresholds (15, 2), the 4 px
    residual drop at iterations 5 and 10 (sticky), 11 LM iterations.  At every
    extraction the masks and compaction maps equal, bit for bit, the oracle's
    extraction of the same state with the same drop history; the trajectory
    matches the oracle's segment by segment (the oracle restarted from the GPU
    state, damping and drop bits at each drop)."""
    sc = scenes.make_scene("large")
    opt = dict(min_cam_obs=15, min_pt_obs=2, drop_residual_px=4.0, extract_every=5)
    gpu = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP32, **opt))
    orc = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(solver=1, **opt))
    alive = np.ones(sc.n_obs, bool)
    rows, table = [], []

    def step():
        # inlier residuals at the state this iteration starts from (the drop's view)
        c, p = gpu.get_params()
        _, res = orc.predicate(c, p)
        r_in = res[~sc.is_outlier]
        table.append((np.sqrt(np.mean(r_in ** 2)), np.mean(r_in > 4.0)))
        return gpu.lm_step()

    for k0, k1 in ((0, 5), (5, 10), (10, 11)):
        cams, pts = gpu.get_params()
        seg = [step()]
        if k0 > 0:
            # this drop iteration's extraction, bit for bit, from the same state and drop history
            geom, res = orc.predicate(cams, pts)
            alive &= ~((geom == 1) & (res > 4.0))
            e = orc.extract((geom.astype(bool) & alive).astype(np.uint8))
            g = gpu.get_active()
            for key in ("cam_mask", "pt_mask", "obs_mask", "cam_rank", "pt_rank"):
                np.testing.assert_array_equal(g[key], e[key], err_msg=f"k={k0} {key}")
        seg += [step() for _ in range(k0 + 1, k1)]
        # the oracle's run of the segment from the same state, damping and drop bits
        # (no drop inside a segment): lambda as logged, nu doubled once per reject
        # since the last accepted step
        rejects = 0
        while rejects < len(rows) and not rows[-1 - rejects]["accepted"]:
            rejects += 1
        orc.opts.lambda0 = seg[0]["lam"]
        orc.opts.nu0 = 2.0 ** (1 + rejects)
        orc.opts.extract_every = 0
        _, _, log_o = orc.lm(cams, pts, k1 - k0, alive=alive.astype(np.uint8).copy())
        for k, (a, o) in enumerate(zip(seg, log_o), start=k0):
            assert a["cost"] == pytest.approx(o["cost"], rel=1e-5), k
            assert a["accepted"] == o["accepted"], k
            assert a["n_obs_act"] == o["n_obs_act"], k
        rows += seg
    om = gpu.get_active()["obs_mask"].astype(bool)
    print("k | cost | active RMSE px | active obs | inlier RMSE px | inliers above 4 px")
    for k, (r, (rin, frac)) in enumerate(zip(rows, table)):
        print(f"{k} | {r['cost']:.4e} | {r['rmse_px']:.3f} | {r['n_obs_act']} | {rin:.3f} | {frac:.4f}")
    print(f"after 11 iterations: kept outliers {om[sc.is_outlier].mean():.4f}, "
          f"inliers {om[~sc.is_outlier].mean():.4f}")
    gpu.close()


def similarity_aligned_errors(p, p_gt):
    """Point errors after the least-squares similarity s R p + t that maps p onto
    p_gt (Umeyama 1991): the error left once the gauge (rotation, translation,
    scale) is taken out, which the depth priors fix only weakly.  The similarity is
    fitted on the points whose raw error is within three times the median (points
    that never rejoin the active set keep gross errors) and applied to all."""
    raw = np.linalg.norm(p - p_gt, axis=1)
    fit = raw <= 3.0 * np.median(raw)
    mu, mu_gt = p[fit].mean(0), p_gt[fit].mean(0)
    a, b = p[fit] - mu, p_gt[fit] - mu_gt
    U, S, Vt = np.linalg.svd(b.T @ a / len(a))
    d = np.ones(3)
    d[2] = np.sign(np.linalg.det(U @ Vt))
    R = U @ np.diag(d) @ Vt
    s = (S * d).sum() / (a * a).sum(1).mean()
    return np.linalg.norm(s * (p - mu) @ R.T + mu_gt - p_gt, axis=1)


def test_extraction_ablation_on_injected_frustum_exits():
    """The ablation idea of Sec. 4.2 (per-iteration extraction against one-shot
    pruning) re-run on the 1M-observation geometry with injected frustum exits
    (30% of the wide points start above the image of their nearer cameras):
    30 FP32 LM iterations in each mode from the same start.  One-shot keeps the
    first active set; dynamic extraction re-admits the observations as the points
    come back into view and ends with more active observations (996,846 against
    908,556).  Point errors are compared after a similarity alignment to the
    ground truth: the raw errors are dominated by drift along the weakly fixed
    gauge, which moves with the rounding of the solves (two formation kernels
    summing in different orders end 30% apart raw and within 0.1% aligned).
    Aligned, dynamic extraction ends with a lower median error on the lifted
    points (measured 2.62e-3 against 3.50e-3) and a slightly higher one over all
    points (2.55e-3 against 2.24e-3).  The table is printed."""
    sc = scenes.make_scene("medium", frustum_exit_frac=0.3)
    lifted = np.flatnonzero(np.abs(sc.pts0[:, 2] - sc.pts_gt[:, 2]) > 0.5)
    res = {}
    for name, mode in (("one-shot", ba.BA_EXTRACT_ONCE), ("dynamic", ba.BA_EXTRACT_DYNAMIC)):
        gpu = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP32, extract_mode=mode))
        log = gpu.solve(30)
        c, p = gpu.get_params()
        gpu.close()
        err = np.linalg.norm(p - sc.pts_gt, axis=1)
        al = similarity_aligned_errors(p, sc.pts_gt)
        res[name] = dict(act0=log[0]["n_obs_act"], act=log[-1]["n_obs_act"], rmse=log[-1]["rmse_px"],
                         rot=pose_diff(c, sc.cams_gt)["rot_deg"], lifted=np.median(err[lifted]),
                         allp=np.median(err), lifted_al=np.median(al[lifted]), allp_al=np.median(al))
    print(f"{len(lifted)} lifted points of {sc.spec.n_pts}")
    print("mode | active obs (first, last) | final RMSE px | max rotation error deg | "
          "median point error: lifted, all | after similarity alignment: lifted, all")
    for k, r in res.items():
        print(f"{k} | {r['act0']}, {r['act']} | {r['rmse']:.3f} | {r['rot']:.4f} | {r['lifted']:.3e}, "
              f"{r['allp']:.3e} | {r['lifted_al']:.3e}, {r['allp_al']:.3e}")
    once, dyn = res["one-shot"], res["dynamic"]
    assert once["act"] == once["act0"] == dyn["act0"]
    assert dyn["act"] > once["act"]
    for r in res.values():
        assert np.isfinite(r["rmse"]) and r["allp_al"] < 1e-2
    assert dyn["lifted_al"] < 0.9 * once["lifted_al"]
