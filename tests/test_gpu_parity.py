"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Each test runs both sides on the same seeded inputs and compares element by
element: step (a)+(b) blocks at an identical state, step (c) masks and ranks
bit for bit, step (d) damped steps, step (e) whole LM trajectories."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2510_13310_b300 import ba, scenes
from parity_util import check_blocks, check_close, check_step

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def tiny(n_cams=8, n_pts=300, track=4, seed=5, **kw):
    spec = dataclasses.replace(scenes.SPECS["small"], n_cams=n_cams, n_pts=n_pts, track_min=track,
                               track_max=track, track_mean=track, seed=seed)
    return scenes.make_scene(spec, **kw)


def geometric(n_cams, n_pts, lo, hi, mean, seed, **kw):
    spec = dataclasses.replace(scenes.SPECS["medium"], n_cams=n_cams, n_pts=n_pts, track_min=lo,
                               track_max=hi, track_mean=mean, seed=seed)
    return scenes.make_scene(spec, **kw)


def pair(scene, precision, **opt):
    o = ba.Options(precision=precision, **opt)
    gpu = ba.Problem.from_scene(scene, o)
    oo = oracle.OracleOptions(**{k: v for k, v in opt.items() if k in oracle.OracleOptions.__dataclass_fields__})
    orc = oracle.OracleBA.from_scene(scene, oo)
    return gpu, orc


# FP64: the GPU and the oracle differ only in summation order (measured <= 2e-8
# of the kind scale for the PCG-to-1e-10 steps).  FP32: products and sums in
# FP32, PCG to 1e-6 (measured <= 4.3e-4 on these scenes).
STEP_TOL = {ba.BA_FP64: (1e-7, 1e-10), ba.BA_FP32: (2e-3, 1e-6)}


# ---------------------------------------------------------------------------
# (a)+(b): normal-equation blocks at an identical state
# ---------------------------------------------------------------------------

# measured worst entries: FP64 ~7e-14 of their scale; FP32 ~2.6e-5 (W)
@pytest.mark.parametrize("precision,tol", [(ba.BA_FP64, 1e-11), (ba.BA_FP32, 1e-4)])
def test_linearization_blocks_match_oracle(precision, tol):
    sc = geometric(12, 3000, 2, 12, 5.0, seed=31)   # several tiles, ragged last tile
    gpu, orc = pair(sc, precision, invalid_depth_weight=1e-3)
    lin = gpu.linearize()
    act = gpu.get_active()
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    np.testing.assert_array_equal(act["obs_mask"], ext["obs_mask"])
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    live = ext["cam_mask"].astype(bool)
    print(check_blocks(lin, ne, orc, sc.cams0, sc.pts0, ext["obs_mask"], live, tol))


def test_cost_fp64_matches_oracle_at_same_state():
    sc = geometric(10, 2000, 2, 10, 5.0, seed=3)
    for prec in (ba.BA_FP64, ba.BA_FP32):
        gpu, orc = pair(sc, prec)
        F, rmse = gpu.eval_cost()
        m = gpu.get_active()["obs_mask"]
        Fo, rmse_o = orc.cost(sc.cams0, sc.pts0, m)
        assert F == pytest.approx(Fo, rel=1e-12)
        assert rmse == pytest.approx(rmse_o, rel=1e-12)
        # another state, passed in
        c2, p2 = sc.cams_gt, sc.pts_gt
        F2, _ = gpu.eval_cost(c2, p2)
        Fo2, _ = orc.cost(c2, p2, m)
        assert F2 == pytest.approx(Fo2, rel=1e-12)


# ---------------------------------------------------------------------------
# (c): extraction masks and ranks, bit for bit
# ---------------------------------------------------------------------------

def _perturb_visibility(sc, rng, n_far=40, n_behind=20):
    """Move some points out of every image and some behind one camera."""
    pts = sc.pts0.copy()
    far = rng.choice(sc.spec.n_pts, n_far, replace=False)
    pts[far] = np.array([0.0, 0.0, 30.0]) + rng.normal(size=(n_far, 3))
    from scipy.spatial.transform import Rotation
    ks = rng.choice(sc.n_obs, n_behind, replace=False)
    for k in ks:
        c = sc.obs_cam[k]
        centre = -Rotation.from_rotvec(sc.cams0[c, :3]).inv().apply(sc.cams0[c, 3:6])
        pts[sc.obs_pt[k]] = 1.02 * centre
    return pts


@pytest.mark.parametrize("thresholds", [(1, 1), (15, 2), (40, 3)])
def test_extraction_bit_exact(thresholds):
    rng = np.random.default_rng(11)
    sc = geometric(30, 4000, 2, 12, 4.0, seed=17)
    pts = _perturb_visibility(sc, rng)
    tc, tp = thresholds
    gpu, orc = pair(sc, ba.BA_FP32, min_cam_obs=tc, min_pt_obs=tp)
    gpu.set_params(sc.cams0, pts)
    gpu.extract()
    g = gpu.get_active()
    geom, _ = orc.predicate(sc.cams0, pts)
    e = orc.extract(geom)
    for key in ("cam_mask", "pt_mask", "obs_mask", "cam_rank", "pt_rank"):
        np.testing.assert_array_equal(g[key], e[key], err_msg=key)
    if thresholds == (1, 1):
        v = geom.astype(bool)
        np.testing.assert_array_equal(np.flatnonzero(g["pt_mask"]), np.unique(sc.obs_pt[v]))


def test_validity_decisions_at_the_threshold_follow_fp64():
    """FP32 problems evaluate in double-float and re-evaluate in FP64 every validity
    decision that falls within rounding of its threshold.  With min_depth 8 ulps
    above or below one observation's FP64 depth (FP64 on both sides decides it the
    same way; double-float alone could not), masks and ranks match the oracle bit
    for bit and that observation gets the FP64 decision."""
    from scipy.spatial.transform import Rotation
    sc = geometric(12, 1500, 2, 8, 4.0, seed=8)
    z = np.array([(Rotation.from_rotvec(sc.cams0[c, :3]).apply(sc.pts0[p]) + sc.cams0[c, 3:6])[2]
                  for c, p in zip(sc.obs_cam, sc.obs_pt)])
    order = np.argsort(z)
    for k in (order[3], order[len(order) // 2]):
        for sign in (-1.0, 1.0):
            md = float(z[k] + sign * 8.0 * np.spacing(z[k]))
            gpu, orc = pair(sc, ba.BA_FP32, min_depth=md)
            gpu.extract()
            g = gpu.get_active()
            geom, _ = orc.predicate(sc.cams0, sc.pts0)
            assert bool(geom[k]) == (sign < 0)
            e = orc.extract(geom)
            for key in ("cam_mask", "pt_mask", "obs_mask", "cam_rank", "pt_rank"):
                np.testing.assert_array_equal(g[key], e[key], err_msg=key)
            gpu.close()


def test_extraction_residual_drop_and_order_invariance():
    sc = geometric(20, 3000, 2, 10, 5.0, seed=23)
    opt = dict(min_cam_obs=15, min_pt_obs=2, drop_residual_px=4.0, extract_every=5)
    gpu, orc = pair(sc, ba.BA_FP32, **opt)
    gpu.extract(drop=True)
    g = gpu.get_active()
    geom, res = orc.predicate(sc.cams0, sc.pts0)
    alive = ~((geom == 1) & (res > 4.0))
    e = orc.extract((geom.astype(bool) & alive).astype(np.uint8))
    for key in ("cam_mask", "pt_mask", "obs_mask", "cam_rank", "pt_rank"):
        np.testing.assert_array_equal(g[key], e[key], err_msg=key)
    # a shuffled observation order gives the same sets
    perm = np.random.default_rng(2).permutation(sc.n_obs)
    sc2 = dataclasses.replace(sc, obs_cam=sc.obs_cam[perm], obs_pt=sc.obs_pt[perm],
                              obs_uv=sc.obs_uv[perm], depth=sc.depth[perm])
    gpu2 = ba.Problem.from_scene(sc2, ba.Options(**opt))
    gpu2.extract(drop=True)
    g2 = gpu2.get_active()
    np.testing.assert_array_equal(g2["pt_mask"], g["pt_mask"])
    np.testing.assert_array_equal(g2["cam_rank"], g["cam_rank"])
    np.testing.assert_array_equal(g2["obs_mask"], g["obs_mask"][perm])


# ---------------------------------------------------------------------------
# (d): damped step (Schur + PCG + back-substitution) vs the oracle's solve
# ---------------------------------------------------------------------------

SOLVERS = [ba.BA_SOLVER_IMPLICIT, ba.BA_SOLVER_EXPLICIT]


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("precision", [ba.BA_FP64, ba.BA_FP32])
def test_damped_step_matches_oracle(precision, solver):
    sc = geometric(12, 3000, 2, 12, 5.0, seed=41)
    gpu, orc = pair(sc, precision, pcg_rel_tol=1e-10 if precision == ba.BA_FP64 else 1e-6,
                    solver=solver)
    lam = 1e-3
    g = gpu.solve_damped(lam)
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    o = orc.solve_step(ne, ext, lam)   # dense Cholesky of the Schur system
    check_step(g, o, *STEP_TOL[precision])
    assert g["pcg_rel_res"] <= (1e-10 if precision == ba.BA_FP64 else 1e-6)
    assert not g["dc"][sc.fixed_cams].any()


@pytest.mark.parametrize("precision,solver", [(ba.BA_FP64, ba.BA_SOLVER_EXPLICIT),
                                              (ba.BA_FP32, ba.BA_SOLVER_EXPLICIT),
                                              (ba.BA_FP32, ba.BA_SOLVER_SPARSE)])
def test_explicit_step_with_many_short_runs_matches_oracle(precision, solver):
    """About 99k co-visible camera pairs of a few shared points each (4 x 128 runs
    per SM and more): FP64 forms the explicit system with one lane per run, FP32
    with the camera-owned formation (owner rows staged in shared memory), into the
    dense and the block-sparse storage."""
    sc = geometric(450, 6000, 12, 12, 12.0, seed=57)
    tracks = np.sort(sc.obs_cam.reshape(-1, 12), axis=1).astype(np.int64)
    iu, ju = np.triu_indices(12, 1)
    n_runs = np.unique(tracks[:, iu] * sc.spec.n_cams + tracks[:, ju]).size
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert n_runs >= 4 * 128 * sms
    gpu, orc = pair(sc, precision, pcg_rel_tol=1e-10 if precision == ba.BA_FP64 else 1e-6, solver=solver)
    lam = 1e-3
    g = gpu.solve_damped(lam)
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    o = orc.solve_step(ne, ext, lam)
    check_step(g, o, *STEP_TOL[precision])


@pytest.mark.parametrize("solver", [ba.BA_SOLVER_IMPLICIT, ba.BA_SOLVER_EXPLICIT, ba.BA_SOLVER_SPARSE,
                                    ba.BA_SOLVER_DENSE])
def test_two_problems_interleaved_on_two_streams(solver):
    """Two problems alive at once, their LM steps and adjoints interleaved on two
    streams, give the same bits as each run alone: no problem reads another's
    state (exchange words, scratch, cached buffers)."""
    a_sc = geometric(30, 4000, 4, 12, 7.0, seed=61)
    b_sc = geometric(45, 6000, 4, 10, 6.0, seed=62)
    o = ba.Options(precision=ba.BA_FP32, solver=solver)

    def alone(sc):
        p = ba.Problem.from_scene(sc, o)
        log = [p.lm_step()["cost"] for _ in range(5)]
        c, q = p.get_params()
        g = p.backward(c - sc.cams_gt, q - sc.pts_gt)
        p.close()
        return log, c, q, g

    ref_a, ref_b = alone(a_sc), alone(b_sc)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    pa = ba.Problem.from_scene(a_sc, o, stream=sa.cuda_stream)
    pb = ba.Problem.from_scene(b_sc, o, stream=sb.cuda_stream)
    la, lb = [], []
    for _ in range(5):
        la.append(pa.lm_step()["cost"])
        lb.append(pb.lm_step()["cost"])
    ca, qa = pa.get_params()
    cb, qb = pb.get_params()
    ga = pa.backward(ca - a_sc.cams_gt, qa - a_sc.pts_gt)
    gb = pb.backward(cb - b_sc.cams_gt, qb - b_sc.pts_gt)
    for got, ref in (((la, ca, qa, ga), ref_a), ((lb, cb, qb, gb), ref_b)):
        assert got[0] == ref[0]
        np.testing.assert_array_equal(got[1], ref[1])
        np.testing.assert_array_equal(got[2], ref[2])
        np.testing.assert_array_equal(got[3][0], ref[3][0])
        np.testing.assert_array_equal(got[3][1], ref[3][1])
    pa.close()
    pb.close()


@pytest.mark.parametrize("solver", [ba.BA_SOLVER_EXPLICIT, ba.BA_SOLVER_IMPLICIT])
def test_reused_device_buffers_give_identical_runs(solver):
    """ba_destroy hands a problem's buffers to the process cache and the next
    ba_create takes them back with the previous problem's contents: the runs must
    not depend on that (no buffer is read before it is written)."""
    sc = geometric(12, 3000, 2, 12, 5.0, seed=41)
    def run():
        p = ba.Problem.from_scene(sc, ba.Options(solver=solver))
        log = [p.lm_step()["cost"] for _ in range(6)]
        cams, pts = p.get_params()
        p.close()
        return log, cams, pts
    first = run()
    other = ba.Problem.from_scene(geometric(12, 3000, 2, 12, 5.0, seed=7), ba.Options(solver=solver))
    other.lm_step()
    other.close()  # its buffers, now dirty, go back to the cache
    second = run()
    ba.release_cache()
    third = run()
    for r in (second, third):
        assert r[0] == first[0]
        assert np.array_equal(r[1], first[1]) and np.array_equal(r[2], first[2])


def test_auto_solver_choice_follows_the_cost_model():
    """AUTO: the explicit system whenever 9 C <= 4608; above that, the per-step cost
    model (formation + streamed S^ against the implicit matvec).  A scene of 700
    cameras with tracks of 2-4 has few co-visible pairs but a 6,300-order S^ whose
    streaming costs more per iteration than the implicit matvec over 20k
    observations: implicit."""
    small = ba.Problem.from_scene(geometric(40, 3000, 2, 10, 5.0, seed=5), ba.Options())
    assert small.solver_kind == ba.BA_SOLVER_EXPLICIT and small.explicit_layout["rows_in_smem"] == 1
    sparse = ba.Problem.from_scene(geometric(700, 8000, 2, 4, 3.0, seed=6), ba.Options())
    assert sparse.solver_kind == ba.BA_SOLVER_IMPLICIT
    assert sparse.explicit_layout == {"rows_in_smem": 0, "vecs_in_smem": 0, "grid": 0}
    small.close()
    sparse.close()


@pytest.mark.parametrize("precision,n_cams", [(ba.BA_FP64, 400), (ba.BA_FP32, 700)])
def test_explicit_solver_vectors_in_global_scratch(precision, n_cams):
    # systems of 3,591 (FP64) and 6,291 (FP32) unknowns: the explicit PCG keeps p
    # in shared memory and its other per-block vectors in global scratch
    sc = geometric(n_cams, 6000, 2, 10, 4.0, seed=77)
    gpu, orc = pair(sc, precision, pcg_rel_tol=1e-10 if precision == ba.BA_FP64 else 1e-6,
                    solver=ba.BA_SOLVER_EXPLICIT, pcg_max_iters=2000)
    assert gpu.explicit_solver
    lam = 1e-3
    g = gpu.solve_damped(lam)
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    o = orc.solve_step(ne, ext, lam)
    check_step(g, o, *STEP_TOL[precision])
    assert g["pcg_rel_res"] <= (1e-10 if precision == ba.BA_FP64 else 1e-6)


# ---------------------------------------------------------------------------
# (e): LM trajectories
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("solver", SOLVERS)
def test_small_scene_fp64_trajectory_matches_oracle(solver):
    """The FP64 small workload: 20 cameras, 2k points, ~20k observations, 10 iterations."""
    sc = scenes.make_scene("small")
    gpu, orc = pair(sc, ba.BA_FP64, solver=solver)
    log_g = gpu.solve(10)
    orc.opts.solver = 1
    c_o, p_o, log_o = orc.lm(sc.cams0, sc.pts0, 10)
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i
        assert a["accepted"] == b["accepted"], i
        assert a["n_obs_act"] == b["n_obs_act"]
    c_g, p_g = gpu.get_params()
    assert np.abs(p_g - p_o).max() < 1e-5
    assert np.abs(c_g - c_o).max() < 1e-4


@pytest.mark.parametrize("solver", SOLVERS)
def test_fp32_trajectory_close_to_oracle(solver):
    sc = geometric(40, 20000, 3, 20, 10.0, seed=1001)
    gpu, orc = pair(sc, ba.BA_FP32, solver=solver)
    log_g = gpu.solve(8)
    orc.opts.solver = 1
    _, _, log_o = orc.lm(sc.cams0, sc.pts0, 8)
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i


def test_inactive_parameters_unchanged_by_a_step():
    rng = np.random.default_rng(4)
    sc = geometric(12, 1500, 2, 8, 4.0, seed=8)
    pts = _perturb_visibility(sc, rng, n_far=30, n_behind=0)
    gpu = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP64))
    gpu.set_params(sc.cams0, pts)
    gpu.lm_step()
    act = gpu.get_active()
    _, p1 = gpu.get_params()
    off = act["pt_mask"] == 0
    assert off.sum() >= 30
    np.testing.assert_array_equal(p1[off], pts[off])


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_invalid_inputs_rejected():
    sc = tiny()
    bad = sc.obs_cam.copy()
    bad[3] = 99
    with pytest.raises(ba.BAError, match="invalid argument"):
        ba.Problem(sc.cams0, sc.pts0, bad, sc.obs_pt, sc.obs_uv, sc.depth)
    dup_c = np.concatenate([sc.obs_cam, sc.obs_cam[:1]])
    dup_p = np.concatenate([sc.obs_pt, sc.obs_pt[:1]])
    with pytest.raises(ba.BAError, match="invalid argument"):
        ba.Problem(sc.cams0, sc.pts0, dup_c, dup_p, np.concatenate([sc.obs_uv, sc.obs_uv[:1]]),
                   np.concatenate([sc.depth, sc.depth[:1]]))
    uv = sc.obs_uv.copy()
    uv[0, 0] = np.nan
    with pytest.raises(ba.BAError, match="invalid argument"):
        ba.Problem(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, uv, sc.depth)


def test_track_length_limit():
    # a point seen by 256 cameras is accepted, 257 is refused
    C = 257
    cams = np.tile(np.array([0, 0, 0, 0, 0, 3.0, 500, 0, 0]), (C, 1))
    cams[:, 0] = np.linspace(-0.1, 0.1, C)
    for n in (256, 257):
        oc = np.arange(n, dtype=np.int32)
        op = np.zeros(n, np.int32)
        uv = np.full((n, 2), 320.0)
        if n == 256:
            p = ba.Problem(cams, np.zeros((1, 3)), oc, op, uv, np.zeros(n))
            p.lm_step()
        else:
            with pytest.raises(ba.BAError, match="invalid argument"):
                ba.Problem(cams, np.zeros((1, 3)), oc, op, uv, np.zeros(n))


@pytest.mark.parametrize("precision,solver", [(ba.BA_FP64, ba.BA_SOLVER_AUTO), (ba.BA_FP64, ba.BA_SOLVER_IMPLICIT),
                                              (ba.BA_FP32, ba.BA_SOLVER_IMPLICIT), (ba.BA_FP32, ba.BA_SOLVER_EXPLICIT),
                                              (ba.BA_FP32, ba.BA_SOLVER_SPARSE), (ba.BA_FP32, ba.BA_SOLVER_DENSE)])
def test_degenerate_problems(precision, solver):
    """Under every solver: only the gauge camera (no camera unknowns), cameras and
    points without observations (LM steps and the adjoint), no observations at
    all; what has no observation stays unchanged."""
    o = ba.Options(precision=precision, solver=solver)
    # only the gauge camera: nothing to solve for cameras, points still move
    sc = tiny(n_cams=4, n_pts=50, track=3, seed=2)
    keep = sc.obs_cam == 0
    p = ba.Problem(sc.cams0[:1], sc.pts0, sc.obs_cam[keep], sc.obs_pt[keep], sc.obs_uv[keep],
                   sc.depth[keep], o)
    info = p.lm_step()
    assert info["pcg_iters"] == 0
    p.close()
    # points and cameras without any observation
    cams = np.concatenate([sc.cams0, sc.cams0[:2]])
    pts = np.concatenate([sc.pts0, np.zeros((5, 3))])
    p = ba.Problem(cams, pts, sc.obs_cam, sc.obs_pt, sc.obs_uv, sc.depth, o)
    p.solve(2)
    act = p.get_active()
    assert not act["cam_mask"][-2:].any() and not act["pt_mask"][-5:].any()
    assert (act["pt_rank"][-5:] == -1).all()
    c, q = p.get_params()
    np.testing.assert_array_equal(c[-2:], cams[-2:])
    np.testing.assert_array_equal(q[-5:], pts[-5:])
    duv, dd = p.backward(c - np.concatenate([sc.cams_gt, sc.cams_gt[:2]]), np.zeros_like(q))
    assert np.all(np.isfinite(duv)) and np.all(np.isfinite(dd))
    p.close()
    # no observations at all
    p = ba.Problem(sc.cams0, sc.pts0, np.zeros(0, np.int32), np.zeros(0, np.int32),
                   np.zeros((0, 2)), np.zeros(0), o)
    info = p.lm_step()
    assert info["n_obs_act"] == 0
    duv, dd = p.backward(np.ones_like(sc.cams0), np.ones_like(sc.pts0))
    assert duv.shape == (0, 2) and dd.shape == (0,)
    p.close()


def test_device_and_host_buffers_agree():
    sc = tiny()
    dev = lambda a: torch.as_tensor(a).cuda()
    p1 = ba.Problem.from_scene(sc)
    p2 = ba.Problem(dev(sc.cams0), dev(sc.pts0), dev(sc.obs_cam), dev(sc.obs_pt), dev(sc.obs_uv),
                    dev(sc.depth))
    l1 = p1.solve(3)
    l2 = p2.solve(3)
    # every reduction runs in a fixed order: the same inputs give bit-identical runs
    assert [a["cost"] for a in l1] == [b["cost"] for b in l2]
    c_dev = torch.zeros((sc.spec.n_cams, 9), dtype=torch.float64, device="cuda")
    p_dev = torch.zeros((sc.spec.n_pts, 3), dtype=torch.float64, device="cuda")
    p2.get_params(c_dev, p_dev)
    c_h, p_h = p1.get_params()
    np.testing.assert_array_equal(c_dev.cpu().numpy(), c_h)
    np.testing.assert_array_equal(p_dev.cpu().numpy(), p_h)


@pytest.mark.parametrize("solver", [ba.BA_SOLVER_IMPLICIT, ba.BA_SOLVER_EXPLICIT])
def test_layout_independent_of_host_threads(monkeypatch, solver):
    # the orderings, tile records and co-visibility runs built by ba_create on
    # host threads give bit-identical runs with one thread and with many
    sc = geometric(40, 6000, 2, 60, 6.0, seed=41)  # long and short tracks, many tiles
    opts = ba.Options(precision=ba.BA_FP32, solver=solver, min_cam_obs=15, min_pt_obs=3)
    runs = []
    for n in ("1", "7"):
        monkeypatch.setenv("BA_HOST_THREADS", n)
        p = ba.Problem.from_scene(sc, opts)
        log = p.solve(3)
        runs.append(([r["cost"] for r in log], p.get_params(), p.get_active()))
        p.close()
    (c1, (cam1, pt1), a1), (c2, (cam2, pt2), a2) = runs
    assert c1 == c2
    np.testing.assert_array_equal(cam1, cam2)
    np.testing.assert_array_equal(pt1, pt2)
    for key in a1:
        np.testing.assert_array_equal(a1[key], a2[key], err_msg=key)


# ---------------------------------------------------------------------------
# (d) with the dense solver: tensor-core Cholesky + preconditioned CG (FP32)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n_cams,n_pts,track", [(40, 3000, 30), (150, 8000, 40)])
def test_dense_solver_damped_step_matches_oracle(n_cams, n_pts, track):
    """Densely co-visible scenes: 40 cameras (one 384-wide factor, 3 tiles) and 150
    cameras (n = 1341: 11 tiles, two 1024-column panels)."""
    sc = geometric(n_cams, n_pts, track, track, float(track), seed=77)
    gpu, orc = pair(sc, ba.BA_FP32, solver=ba.BA_SOLVER_DENSE)
    assert gpu.explicit_solver is False and ba.lib().ba_solver_kind(gpu.h) == ba.BA_SOLVER_DENSE
    lam = 1e-3
    g = gpu.solve_damped(lam)
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    o = orc.solve_step(ne, ext, lam)
    check_step(g, o, *STEP_TOL[ba.BA_FP32])
    assert g["pcg_rel_res"] <= 1e-6
    # the factor is a good preconditioner: CG needs only a few iterations
    assert g["pcg_iters"] <= 20


def test_dense_solver_trajectory_close_to_oracle():
    sc = geometric(40, 3000, 30, 30, 30.0, seed=78)
    gpu, orc = pair(sc, ba.BA_FP32, solver=ba.BA_SOLVER_DENSE)
    log_g = gpu.solve(8)
    orc.opts.solver = 1
    _, _, log_o = orc.lm(sc.cams0, sc.pts0, 8)
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i


def test_dense_solver_rejects_fp64():
    sc = tiny()
    with pytest.raises(ba.BAError):
        ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP64, solver=ba.BA_SOLVER_DENSE))


def test_explicit_solver_with_many_short_runs_matches_oracle():
    """600 cameras sharing a few points per camera pair: ~170k co-visibility runs of
    ~5 pairs, formed with one lane per run."""
    sc = geometric(600, 30000, 8, 8, 8.0, seed=79)
    gpu, orc = pair(sc, ba.BA_FP32, solver=ba.BA_SOLVER_EXPLICIT)
    lam = 1e-3
    g = gpu.solve_damped(lam)
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    o = orc.solve_step(ne, ext, lam)
    check_step(g, o, *STEP_TOL[ba.BA_FP32])


@pytest.mark.parametrize("solver", [ba.BA_SOLVER_EXPLICIT, ba.BA_SOLVER_SPARSE])
@pytest.mark.parametrize("model", [ba.BA_CAMERA_RADIAL, ba.BA_CAMERA_CENTRE])
def test_formation_from_records_and_from_rows_match_oracle(monkeypatch, solver, model):
    """FP32 explicit systems with a few hundred pairs per camera pair: the blocks
    formed from the observation records (k_form_S_rec: D, the rotated point, the
    normalised point, the weight; V*^-1 per point) and from the Y^ rows
    (k_form_S_runs, selected by BA_FORM_RECORDS=0) both give the oracle's damped
    step, under both camera models and both storages, and each is deterministic."""
    sc = geometric(30, 8000, 3, 14, 8.0, seed=91, camera_model="centre" if model == ba.BA_CAMERA_CENTRE else "radial")
    lam = 1e-3
    steps = {}
    for env in ("1", "0"):
        monkeypatch.setenv("BA_FORM_RECORDS", env)
        gpu, orc = pair(sc, ba.BA_FP32, solver=solver, camera_model=model)
        steps[gpu.formation_kernel] = gpu.solve_damped(lam)
        again = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP32, solver=solver, camera_model=model))
        g2 = again.solve_damped(lam)
        assert np.array_equal(g2["dc"], steps[gpu.formation_kernel]["dc"])
        gpu.close(); again.close()
    assert set(steps) == {"k_form_S_rec", "k_form_S_runs"}
    o = _oracle_step_model(sc, orc, lam)
    for g in steps.values():
        check_step(g, o, *STEP_TOL[ba.BA_FP32])


def _oracle_step_model(sc, orc, lam):
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    return orc.solve_step(ne, ext, lam)


# ---------------------------------------------------------------------------
# checkpoint / resume
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision,solver", [(ba.BA_FP32, ba.BA_SOLVER_EXPLICIT), (ba.BA_FP32, ba.BA_SOLVER_IMPLICIT),
                                              (ba.BA_FP64, ba.BA_SOLVER_EXPLICIT)])
def test_checkpoint_resume_repeats_the_run_bit_for_bit(precision, solver):
    """A run with residual drops (iterations 3, 6) checkpointed after 4 iterations and
    resumed, in a fresh problem and in the original one, repeats the uninterrupted
    run exactly: every reduction has a fixed order."""
    sc = geometric(20, 3000, 2, 10, 5.0, seed=23)
    o = ba.Options(precision=precision, solver=solver, extract_every=3, drop_residual_px=4.0,
                   min_cam_obs=5, min_pt_obs=2, fixed_cams=tuple(sc.fixed_cams))
    p = ba.Problem.from_scene(sc, o)
    p.solve(4)
    blob = p.get_state()
    tail = p.solve(4)
    c_end, p_end = p.get_params()
    for q in (ba.Problem.from_scene(sc, o), p):
        q.set_state(blob)
        tail2 = q.solve(4)
        c2, p2 = q.get_params()
        assert [r["cost"] for r in tail2] == [r["cost"] for r in tail]
        assert [r["accepted"] for r in tail2] == [r["accepted"] for r in tail]
        assert [r["n_obs_act"] for r in tail2] == [r["n_obs_act"] for r in tail]
        assert np.array_equal(c2, c_end) and np.array_equal(p2, p_end)
    # a blob does not load into a problem built from other observations
    other = ba.Problem.from_scene(geometric(20, 3000, 2, 10, 5.0, seed=24), o)
    with pytest.raises(ba.BAError):
        other.set_state(blob)


# ---------------------------------------------------------------------------
# one-shot pruning vs dynamic extraction (Sec. 4.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [ba.BA_EXTRACT_ONCE, ba.BA_EXTRACT_DYNAMIC])
def test_extraction_mode_trajectory_matches_oracle(mode):
    """Injected frustum exits (points starting above the image of their nearer
    cameras).  One-shot pruning keeps the first active set, bit for bit the
    oracle's extraction at the start; dynamic extraction re-admits observations
    as the points come back.  Both follow the oracle's costs per iteration."""
    sc = scenes.make_scene("small", frustum_exit_frac=0.3)
    gpu, orc = pair(sc, ba.BA_FP32, extract_mode=mode)
    log_g = gpu.solve(10)
    _, _, log_o = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(solver=1, extract_mode=mode)).lm(
        sc.cams0, sc.pts0, 10)
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i
        assert a["accepted"] == b["accepted"], i
        assert a["n_obs_act"] == b["n_obs_act"], i
    acts = [r["n_obs_act"] for r in log_g]
    if mode == ba.BA_EXTRACT_ONCE:
        assert len(set(acts)) == 1
        geom, _ = orc.predicate(sc.cams0, sc.pts0)
        e = orc.extract(geom)
        g = gpu.get_active()
        for key in ("cam_mask", "pt_mask", "obs_mask", "cam_rank", "pt_rank"):
            np.testing.assert_array_equal(g[key], e[key], err_msg=key)
    else:
        assert acts[-1] > acts[0]


# ---------------------------------------------------------------------------
# (d) with the block-sparse explicit system (sparse co-visibility)
# ---------------------------------------------------------------------------

def window_scene(n_cams, n_pts, lo, hi, mean, seed, **kw):
    spec = dataclasses.replace(scenes.SPECS["window"], n_cams=n_cams, n_pts=n_pts, track_min=lo,
                               track_max=hi, track_mean=mean, seed=seed)
    return scenes.make_scene(spec, covis="window", **kw)


@pytest.mark.parametrize("precision", [ba.BA_FP64, ba.BA_FP32])
def test_sparse_solver_damped_step_matches_oracle(precision):
    """Windowed tracks (each point seen by the cameras nearest its azimuth): a
    block-banded reduced camera system stored as the 9x9 blocks of its co-visible
    camera pairs; the damped step against the oracle's dense Cholesky solve."""
    sc = window_scene(120, 12000, 3, 10, 6.0, seed=91)
    gpu, orc = pair(sc, precision, pcg_rel_tol=1e-10 if precision == ba.BA_FP64 else 1e-6,
                    solver=ba.BA_SOLVER_SPARSE, pcg_max_iters=2000)
    assert gpu.solver_kind == ba.BA_SOLVER_SPARSE
    lam = 1e-3
    g = gpu.solve_damped(lam)
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    o = orc.solve_step(ne, ext, lam)
    check_step(g, o, *STEP_TOL[precision])
    assert g["pcg_rel_res"] <= (1e-10 if precision == ba.BA_FP64 else 1e-6)


def test_sparse_solver_trajectory_and_extraction_match_oracle():
    """LM iterations with the block-sparse system follow the oracle per iteration,
    also when extraction removes cameras (thresholds (15, 2) and a residual drop):
    blocks of pairs whose cameras left the solve are skipped by the matvec.  FP64:
    the narrow baselines of windowed tracks make the FP32 steps differ from the
    FP64 ones by more than the 1e-5 cost bar (the FP32 steps are checked above)."""
    sc = window_scene(80, 8000, 3, 10, 6.0, seed=92)
    opt = dict(min_cam_obs=15, min_pt_obs=2, drop_residual_px=4.0, extract_every=3)
    gpu, orc = pair(sc, ba.BA_FP64, solver=ba.BA_SOLVER_SPARSE, pcg_rel_tol=1e-10, pcg_max_iters=2000, **opt)
    log_g = gpu.solve(8)
    orc.opts.solver = 1
    _, _, log_o = orc.lm(sc.cams0, sc.pts0, 8)
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i
        assert a["accepted"] == b["accepted"], i
        assert a["n_obs_act"] == b["n_obs_act"], i


def test_sparse_and_dense_explicit_agree_and_auto_prefers_sparse():
    """The block-sparse and the dense explicit systems hold the same blocks: their
    damped steps agree to FP32 rounding of the PCG.  On a windowed scene with many
    cameras, AUTO prices the block-sparse system cheapest."""
    sc = window_scene(150, 15000, 3, 10, 6.0, seed=93)
    steps = []
    for solver in (ba.BA_SOLVER_SPARSE, ba.BA_SOLVER_EXPLICIT):
        p = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP64, solver=solver, pcg_rel_tol=1e-12,
                                                 pcg_max_iters=3000))
        steps.append(p.solve_damped(1e-3))
        p.close()
    check_step(steps[0], steps[1], 1e-8, 1e-10)
    big = window_scene(900, 60000, 3, 10, 6.0, seed=94)
    p = ba.Problem.from_scene(big, ba.Options())
    assert p.solver_kind == ba.BA_SOLVER_SPARSE
    p.close()


# ---------------------------------------------------------------------------
# the camera parameterisation of Sec. 3.2 (BA_CAMERA_CENTRE)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision,tol", [(ba.BA_FP64, 1e-11), (ba.BA_FP32, 1e-4)])
def test_centre_model_blocks_match_oracle(precision, tol):
    sc = geometric(12, 3000, 2, 12, 5.0, seed=31, camera_model="centre")
    gpu, orc = pair(sc, precision, camera_model=ba.BA_CAMERA_CENTRE, solver=ba.BA_SOLVER_EXPLICIT)
    lin = gpu.linearize()
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    np.testing.assert_array_equal(gpu.get_active()["obs_mask"], ext["obs_mask"])
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    print(check_blocks(lin, ne, orc, sc.cams0, sc.pts0, ext["obs_mask"], ext["cam_mask"].astype(bool), tol))
    assert not lin["U"][:, 7:, :].any() and not lin["W"][:, 7:, :].any()  # no distortion rows


@pytest.mark.parametrize("precision,solver", [(ba.BA_FP64, ba.BA_SOLVER_IMPLICIT),
                                              (ba.BA_FP64, ba.BA_SOLVER_EXPLICIT),
                                              (ba.BA_FP32, ba.BA_SOLVER_IMPLICIT),
                                              (ba.BA_FP32, ba.BA_SOLVER_EXPLICIT),
                                              (ba.BA_FP32, ba.BA_SOLVER_SPARSE)])
def test_centre_model_damped_step_matches_oracle(precision, solver):
    """The damped step under every solver; the FP32 implicit PCG recomputes the
    centre model's blocks inside its matvec (rotation columns on R (X - c), centre
    columns -D R, no distortion columns)."""
    sc = geometric(12, 3000, 2, 12, 5.0, seed=41, camera_model="centre")
    gpu, orc = pair(sc, precision, camera_model=ba.BA_CAMERA_CENTRE, solver=solver,
                    pcg_rel_tol=1e-10 if precision == ba.BA_FP64 else 1e-6)
    lam = 1e-3
    g = gpu.solve_damped(lam)
    geom, _ = orc.predicate(sc.cams0, sc.pts0)
    ext = orc.extract(geom)
    ne = orc.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    o = orc.solve_step(ne, ext, lam)
    check_step(g, o, *STEP_TOL[precision])
    assert not g["dc"][:, 7:].any()


def test_centre_model_trajectory_and_restrictions():
    """FP32 LM with the centre model follows the oracle per iteration, with the
    explicit and with the implicit solver; the allocation-free cost follows the
    model too."""
    sc = geometric(40, 20000, 3, 20, 10.0, seed=1001, camera_model="centre")
    gpu, orc = pair(sc, ba.BA_FP32, camera_model=ba.BA_CAMERA_CENTRE)
    assert gpu.solver_kind == ba.BA_SOLVER_EXPLICIT
    log_g = gpu.solve(8)
    orc.opts.solver = 1
    c_o, p_o, log_o = orc.lm(sc.cams0, sc.pts0, 8)
    for i, (a, b) in enumerate(zip(log_g, log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i
        assert a["accepted"] == b["accepted"], i
    c_g, _ = gpu.get_params()
    np.testing.assert_array_equal(c_g[:, 7:], sc.cams0[:, 7:])  # k1, k2 untouched
    imp = ba.Problem.from_scene(sc, ba.Options(precision=ba.BA_FP32, camera_model=ba.BA_CAMERA_CENTRE,
                                               solver=ba.BA_SOLVER_IMPLICIT))
    for i, (a, b) in enumerate(zip(imp.solve(8), log_o)):
        assert a["cost"] == pytest.approx(b["cost"], rel=1e-5), i
        assert a["accepted"] == b["accepted"], i
    imp.close()
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    ba.eval_cost_noalloc(dev(sc.cams_gt, torch.float64), dev(sc.pts_gt, torch.float64),
                         dev(sc.obs_cam, torch.int32), dev(sc.obs_pt, torch.int32),
                         dev(sc.obs_uv, torch.float64), dev(sc.depth, torch.float64), out,
                         options=ba.Options(camera_model=ba.BA_CAMERA_CENTRE))
    torch.cuda.synchronize()
    F_o, _ = orc.cost(sc.cams_gt, sc.pts_gt)
    assert out[0].item() == pytest.approx(F_o, rel=1e-12)
