"""Pins of the FP64 CPU oracle against things the paper and the mathematics fix.

None of these re-types an oracle formula: each checks the oracle against an
independent route (SciPy rotations, central finite differences, a dense NumPy
solve of the full damped system, np.unique / searchsorted, brute-force subset
enumeration, closed forms, invariances, exact convergence)."""
import dataclasses
import itertools
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2510_13310_b300 import scenes


def tiny_scene(n_cams=5, n_pts=30, track=3, seed=7, **kw):
    spec = dataclasses.replace(scenes.SPECS["small"], n_cams=n_cams, n_pts=n_pts,
                               track_min=track, track_max=track, track_mean=track, seed=seed)
    return scenes.make_scene(spec, **kw)


# --------------------------------------------------------------------------
# rotations and the camera model (Sec. 3.2)
# --------------------------------------------------------------------------

def test_rotation_matches_scipy():
    rng = np.random.default_rng(0)
    ws = [np.zeros(3), np.array([1e-10, -2e-10, 0.5e-10]), np.array([0.0, 0.0, math.pi]),
          np.array([math.pi - 1e-9, 0, 0])] + [rng.normal(size=3) for _ in range(20)]
    for w in ws:
        np.testing.assert_allclose(oracle.rotvec_to_matrix(w),
                                   Rotation.from_rotvec(w).as_matrix(), atol=1e-13)
    for _ in range(20):
        a, b = rng.normal(size=3) * 0.3, rng.normal(size=3)
        got = Rotation.from_rotvec(oracle.rotvec_compose(a, b)).as_matrix()
        ref = (Rotation.from_rotvec(a) * Rotation.from_rotvec(b)).as_matrix()
        np.testing.assert_allclose(got, ref, atol=1e-13)


def test_projection_closed_forms():
    # w = 0, k1 = k2 = 0: pinhole u = f X/Z + cx
    X = np.array([0.3, -0.2, 2.5])
    cam = np.array([0, 0, 0, 0.1, 0.05, 0.5, 480.0, 0, 0])
    r, _, _, z, uvh = oracle.observe(cam, X, np.zeros(2), 0.0, 0.0)
    P = X + cam[3:6]
    assert z == pytest.approx(P[2], abs=1e-15)
    np.testing.assert_allclose(uvh, [480 * P[0] / P[2] + 320, 480 * P[1] / P[2] + 240], atol=1e-12)
    # quarter turn about z: (x, y, z) -> (-y, x, z); radial distortion applied to rr
    cam = np.array([0, 0, math.pi / 2, 0, 0, 0, 500.0, 0.1, -0.05])
    r, _, _, z, uvh = oracle.observe(cam, X, np.zeros(2), 0.0, 0.0)
    xn, yn = -X[1] / X[2], X[0] / X[2]
    rr = xn * xn + yn * yn
    d = 1 + 0.1 * rr - 0.05 * rr * rr
    np.testing.assert_allclose(uvh, [500 * d * xn + 320, 500 * d * yn + 240], atol=1e-11)


def test_depth_residual_and_mask():
    """Sec. 4.1: r_d = 1/Depth - m/d; m = 0 entries carry the invalid-depth weight."""
    X = np.array([0.1, 0.2, 3.0])
    cam = np.array([0, 0, 0, 0, 0, 1.0, 500.0, 0, 0])
    z = 4.0
    r, Jc, Jp, _, _ = oracle.observe(cam, X, np.zeros(2), 1 / 3.9, 2.0)
    assert r[2] == pytest.approx(math.sqrt(2.0) * (1 / z - 1 / 3.9), rel=1e-14)
    # no prior, zero weight: the row vanishes entirely
    r, Jc, Jp, _, _ = oracle.observe(cam, X, np.zeros(2), 0.0, 0.0)
    assert r[2] == 0.0 and not Jc[2].any() and not Jp[2].any()
    # no prior, sentinel weight: weak prior pulling 1/z to 0
    r, _, _, _, _ = oracle.observe(cam, X, np.zeros(2), 0.0, 1e-3)
    assert r[2] == pytest.approx(math.sqrt(1e-3) / z, rel=1e-14)


def test_huber_closed_form():
    """rho(s) = s for s <= delta^2 else 2 delta sqrt(s) - delta^2; F = 1/2 sum rho."""
    X = np.array([[0.0, 0.0, 2.0]])
    cams = np.array([[0, 0, 0, 0, 0, 0, 500.0, 0, 0]])
    for du, delta, expect in [(0.5, 1.0, 0.25), (3.0, 1.0, 5.0), (3.0, 2.0, 8.0), (3.0, 0.0, 9.0)]:
        ob = oracle.OracleBA(1, 1, [0], [0], [[320.0 + du, 240.0]], [0.0], fixed_cams=[],
                             opts=oracle.OracleOptions(huber_delta=delta))
        F, _ = ob.cost(cams, X)
        assert F == pytest.approx(0.5 * expect, rel=1e-14)


# --------------------------------------------------------------------------
# Jacobians (Eq. LM: J = dr/dtheta) against central finite differences
# --------------------------------------------------------------------------

def _perturb_cam(cam, i, h):
    c = cam.copy()
    if i < 3:
        e = np.zeros(3)
        e[i] = h
        c[:3] = (Rotation.from_rotvec(e) * Rotation.from_rotvec(cam[:3])).as_rotvec()
    else:
        c[i] += h
    return c


def test_jacobian_central_fd():
    rng = np.random.default_rng(1)
    for trial in range(40):
        cam = np.concatenate([rng.normal(size=3) * 0.7, rng.normal(size=3) * 0.3 + [0, 0, 3],
                              [500 + 20 * rng.normal(), 0.05 * rng.normal(), 0.05 * rng.normal()]])
        X = rng.normal(size=3) * 0.5
        uv = rng.uniform(0, 600, 2)
        tau, wt = (1 / 3.1, 1.0) if trial % 2 else (0.0, 0.25)
        r0, Jc, Jp, _, _ = oracle.observe(cam, X, uv, tau, wt)
        h = 1e-6
        for i in range(9):
            rp = oracle.observe(_perturb_cam(cam, i, h), X, uv, tau, wt)[0]
            rm = oracle.observe(_perturb_cam(cam, i, -h), X, uv, tau, wt)[0]
            fd = (rp - rm) / (2 * h)
            np.testing.assert_allclose(Jc[:, i], fd, rtol=1e-7, atol=1e-7 * max(1.0, np.abs(fd).max()))
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            fd = (oracle.observe(cam, X + e, uv, tau, wt)[0] - oracle.observe(cam, X - e, uv, tau, wt)[0]) / (2 * h)
            np.testing.assert_allclose(Jp[:, i], fd, rtol=1e-7, atol=1e-7 * max(1.0, np.abs(fd).max()))


# --------------------------------------------------------------------------
# normal equations, Schur complement and the damped step vs a dense solve
# --------------------------------------------------------------------------

def _dense_system(ob, cams, pts, mask, ext):
    """Dense J (stacked, robust-weighted) over the compacted unknowns, built from
    central finite differences of the oracle's residuals."""
    C, P = ob.n_cams, ob.n_pts
    free = [c for c in range(C) if ext["cam_rank"][c] >= 0]
    act = [p for p in range(P) if ext["pt_rank"][p] >= 0]
    cols = [("c", c, i) for c in free for i in range(9)] + [("p", p, i) for p in act for i in range(3)]
    base = ob.eval_obs(cams, pts, want_jac=False)["r"]
    s = (base ** 2).sum(1)
    delta = ob.opts.huber_delta
    if delta > 0:
        wrob = np.where(s <= delta ** 2, 1.0, delta / np.sqrt(np.maximum(s, 1e-300))) * mask
    else:
        wrob = mask.astype(np.float64)
    J = np.zeros((ob.n_obs, 3, len(cols)))
    h = 1e-6
    for j, (kind, idx, i) in enumerate(cols):
        if kind == "c":
            cp, cm = cams.copy(), cams.copy()
            cp[idx] = _perturb_cam(cams[idx], i, h)
            cm[idx] = _perturb_cam(cams[idx], i, -h)
            rp = ob.eval_obs(cp, pts, False)["r"]
            rm = ob.eval_obs(cm, pts, False)["r"]
        else:
            pp, pm = pts.copy(), pts.copy()
            pp[idx, i] += h
            pm[idx, i] -= h
            rp = ob.eval_obs(cams, pp, False)["r"]
            rm = ob.eval_obs(cams, pm, False)["r"]
        J[:, :, j] = (rp - rm) / (2 * h)
    H = np.einsum("k,kai,kaj->ij", wrob, J, J)
    g = np.einsum("k,kai,ka->i", wrob, J, base)
    return H, g, free, act


def test_normal_equations_and_step_vs_dense():
    sc = tiny_scene(noise=True, outliers=True)
    ob = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(huber_delta=1.0, invalid_depth_weight=1e-3))
    cams, pts = sc.cams0, sc.pts0
    geom, _ = ob.predicate(cams, pts)
    ext = ob.extract(geom)
    mask = ext["obs_mask"]
    ne = ob.normal_equations(cams, pts, mask)
    H, g, free, act = _dense_system(ob, cams, pts, mask, ext)
    nc = 9 * len(free)
    # blocks of the dense matrix vs the oracle's accumulated blocks
    for a, c in enumerate(free):
        blk = H[9 * a:9 * a + 9, 9 * a:9 * a + 9]
        np.testing.assert_allclose(ne["U"][c], blk, rtol=1e-5, atol=1e-5 * np.abs(blk).max())
        np.testing.assert_allclose(ne["gc"][c], g[9 * a:9 * a + 9], rtol=1e-5, atol=1e-5 * np.abs(g).max())
    for b, p in enumerate(act):
        blk = H[nc + 3 * b:nc + 3 * b + 3, nc + 3 * b:nc + 3 * b + 3]
        np.testing.assert_allclose(ne["V"][p], blk, rtol=1e-5, atol=1e-5 * np.abs(blk).max())
    for k in np.flatnonzero(mask):
        c, p = sc.obs_cam[k], sc.obs_pt[k]
        if ext["cam_rank"][c] < 0:
            continue
        a, b = ext["cam_rank"][c], ext["pt_rank"][p]
        blk = H[9 * a:9 * a + 9, nc + 3 * b:nc + 3 * b + 3]
        np.testing.assert_allclose(ne["W"][k], blk, rtol=1e-5, atol=1e-5 * np.abs(H).max())

    # damped full system solved densely vs the oracle's Schur + back-substitution
    lam = 1e-2
    D = np.clip(np.diag(H), 1e-6, 1e32)
    dx = np.linalg.solve(H + lam * np.diag(D), -g)
    for solver in (0, 1):
        ob.opts.solver = solver
        ob.opts.pcg_rel_tol = 1e-12
        st = ob.solve_step(ne, ext, lam)
        assert st["status"] >= 0
        got = np.concatenate([st["dc"][free].ravel(), st["dp"][act].ravel()])
        np.testing.assert_allclose(got, dx, rtol=1e-4, atol=1e-6 * np.abs(dx).max())
        pred = -g @ dx - 0.5 * dx @ H @ dx
        assert st["pred_decrease"] == pytest.approx(pred, rel=1e-4)
        # untouched: gauge camera and inactive entries
        assert not st["dc"][sc.fixed_cams].any()

    # explicit Schur complement = A - B C^-1 B^T of the damped dense matrix
    Hd = H + lam * np.diag(D)
    A, B, Cm = Hd[:nc, :nc], Hd[:nc, nc:], Hd[nc:, nc:]
    S_ref = A - B @ np.linalg.solve(Cm, B.T)
    b_ref = -g[:nc] + B @ np.linalg.solve(Cm, g[nc:])
    S, bb = ob.schur_dense(ne, ext, lam)
    np.testing.assert_allclose(S, S_ref, rtol=1e-4, atol=1e-5 * np.abs(S_ref).max())
    np.testing.assert_allclose(bb, b_ref, rtol=1e-4, atol=1e-5 * np.abs(b_ref).max())


def test_gauss_newton_limit_is_least_squares():
    """lambda -> 0 with no robust loss: the step is the least-squares solution of J dx = -r."""
    sc = tiny_scene(noise=True, outliers=False, seed=11)
    ob = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(huber_delta=0.0))
    geom, _ = ob.predicate(sc.cams0, sc.pts0)
    ext = ob.extract(geom)
    ne = ob.normal_equations(sc.cams0, sc.pts0, ext["obs_mask"])
    H, g, free, act = _dense_system(ob, sc.cams0, sc.pts0, ext["obs_mask"], ext)
    st = ob.solve_step(ne, ext, 1e-12)
    got = np.concatenate([st["dc"][free].ravel(), st["dp"][act].ravel()])
    ref = np.linalg.lstsq(H, -g, rcond=None)[0]
    np.testing.assert_allclose(got, ref, rtol=1e-3, atol=1e-5 * np.abs(ref).max())


# --------------------------------------------------------------------------
# extraction (Sec. 4.2 steps 1-2)
# --------------------------------------------------------------------------

def test_extract_equals_unique_and_rank():
    sc = tiny_scene(n_cams=12, n_pts=200, track=4, seed=3)
    ob = oracle.OracleBA.from_scene(sc)
    rng = np.random.default_rng(5)
    for trial in range(10):
        valid = (rng.random(sc.n_obs) < 0.3 + 0.07 * trial).astype(np.uint8)
        valid[np.flatnonzero(sc.obs_cam == 0)[:1]] = 1  # the gauge camera keeps an observation
        ext = ob.extract(valid)
        v = valid.astype(bool)
        ucam = np.unique(sc.obs_cam[v])
        upt = np.unique(sc.obs_pt[v])
        np.testing.assert_array_equal(np.flatnonzero(ext["cam_mask"]), ucam)
        np.testing.assert_array_equal(np.flatnonzero(ext["pt_mask"]), upt)
        np.testing.assert_array_equal(ext["obs_mask"], valid)
        free = ucam[ucam != 0]
        exp_cr = np.full(sc.spec.n_cams, -1)
        exp_cr[free] = np.searchsorted(free, free)
        np.testing.assert_array_equal(ext["cam_rank"], exp_cr)
        exp_pr = np.full(sc.spec.n_pts, -1)
        exp_pr[upt] = np.searchsorted(upt, upt)
        np.testing.assert_array_equal(ext["pt_rank"], exp_pr)


def _brute_force_peel(C, P, obs_cam, obs_pt, valid, fixed, tc, tp):
    """Largest (cams, pts) pair meeting both thresholds, by enumerating every subset."""
    best = (set(), set())
    vk = [(c, p) for c, p, v in zip(obs_cam, obs_pt, valid) if v]
    for cm in itertools.product([0, 1], repeat=C):
        if any(fixed[c] and not cm[c] for c in range(C)):
            continue
        for pm in itertools.product([0, 1], repeat=P):
            ok = True
            cc = [0] * C
            pc = [0] * P
            for c, p in vk:
                if cm[c] and pm[p]:
                    cc[c] += 1
                    pc[p] += 1
            for c in range(C):
                if cm[c] and not fixed[c] and cc[c] < tc:
                    ok = False
            for p in range(P):
                if pm[p] and pc[p] < tp:
                    ok = False
            if ok:
                s = ({c for c in range(C) if cm[c]}, {p for p in range(P) if pm[p]})
                if len(s[0]) + len(s[1]) > len(best[0]) + len(best[1]):
                    best = s
    return best


def test_peel_is_largest_feasible_subset_and_order_free():
    rng = np.random.default_rng(9)
    for trial in range(6):
        C, P = 4, 7
        pairs = [(c, p) for c in range(C) for p in range(P) if rng.random() < 0.6]
        obs_cam = np.array([c for c, _ in pairs], np.int32)
        obs_pt = np.array([p for _, p in pairs], np.int32)
        valid = (rng.random(len(pairs)) < 0.85).astype(np.uint8)
        tc, tp = 3, 2
        ob = oracle.OracleBA(C, P, obs_cam, obs_pt, np.zeros((len(pairs), 2)), np.zeros(len(pairs)),
                             fixed_cams=[0], opts=oracle.OracleOptions(min_cam_obs=tc, min_pt_obs=tp))
        ext = ob.extract(valid)
        bc, bp = _brute_force_peel(C, P, obs_cam, obs_pt, valid, [1, 0, 0, 0], tc, tp)
        assert set(np.flatnonzero(ext["cam_mask"])) == bc
        assert set(np.flatnonzero(ext["pt_mask"])) == bp
        # shuffling the observation order changes nothing
        perm = rng.permutation(len(pairs))
        ob2 = oracle.OracleBA(C, P, obs_cam[perm], obs_pt[perm], np.zeros((len(pairs), 2)),
                              np.zeros(len(pairs)), fixed_cams=[0], opts=ob.opts)
        ext2 = ob2.extract(valid[perm])
        np.testing.assert_array_equal(ext2["cam_mask"], ext["cam_mask"])
        np.testing.assert_array_equal(ext2["pt_mask"], ext["pt_mask"])
        np.testing.assert_array_equal(ext2["obs_mask"], ext["obs_mask"][perm])


def test_predicate_handcrafted_and_inactive_untouched():
    """Points behind a camera / outside the image are invalid; a point or camera
    left with no valid observation leaves the solve and keeps its value."""
    sc = tiny_scene(n_cams=6, n_pts=40, track=4, seed=21, noise=False, outliers=False)
    pts = sc.pts0.copy()
    cams = sc.cams0.copy()
    # point 0 lifted far above the camera circle: outside every image
    pts[0] = [0.3, 0.2, 40.0]
    # point 1 moved right behind the camera that sees it first
    c1 = sc.obs_cam[np.flatnonzero(sc.obs_pt == 1)[0]]
    centre = -Rotation.from_rotvec(cams[c1, :3]).inv().apply(cams[c1, 3:6])
    pts[1] = 1.05 * centre
    ob = oracle.OracleBA.from_scene(sc)
    geom, _ = ob.predicate(cams, pts)
    R = Rotation.from_rotvec(cams[:, :3]).as_matrix()
    P = np.einsum("kij,kj->ki", R[sc.obs_cam], pts[sc.obs_pt]) + cams[sc.obs_cam, 3:6]
    xn = P[:, 0] / P[:, 2]
    yn = P[:, 1] / P[:, 2]
    rr = xn ** 2 + yn ** 2
    d = 1 + cams[sc.obs_cam, 7] * rr + cams[sc.obs_cam, 8] * rr ** 2
    u = cams[sc.obs_cam, 6] * d * xn + 320
    v = cams[sc.obs_cam, 6] * d * yn + 240
    exp = (P[:, 2] > 0.1) & (u >= 0) & (u < 640) & (v >= 0) & (v < 480)
    np.testing.assert_array_equal(geom.astype(bool), exp)
    assert not geom[sc.obs_pt == 0].any()
    k1 = np.flatnonzero((sc.obs_pt == 1) & (sc.obs_cam == c1))[0]
    assert P[k1, 2] < 0.1 and not geom[k1]
    ext = ob.extract(geom)
    assert ext["pt_mask"][0] == 0 and ext["pt_rank"][0] == -1
    # camera 3 loses every observation
    valid = geom.copy()
    valid[sc.obs_cam == 3] = 0
    ext = ob.extract(valid)
    assert ext["cam_mask"][3] == 0 and ext["cam_rank"][3] == -1
    # one LM iteration: inactive point stays put, inactive camera stays put
    c1, p1, rows = ob.lm(cams, pts, 1)
    np.testing.assert_array_equal(p1[0], pts[0])
    assert rows[0]["n_pt_act"] == sc.spec.n_pts - 1


# --------------------------------------------------------------------------
# whole-loop properties
# --------------------------------------------------------------------------

@pytest.mark.parametrize("depth", [True, False])
def test_noise_free_converges_to_zero(depth):
    sc = scenes.make_scene("small", noise=False, outliers=False, depth_priors=depth)
    ob = oracle.OracleBA.from_scene(sc)
    c, p, rows = ob.lm(sc.cams0, sc.pts0, 20)
    F_end, _ = ob.cost(c, p)
    assert F_end <= 1e-20 * rows[0]["cost"]
    acc = [r["cost"] for r in rows]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(acc, acc[1:]))


def test_similarity_invariance_without_priors():
    sc = scenes.make_scene("small", depth_priors=False)
    ob = oracle.OracleBA.from_scene(sc)
    cams, pts = sc.cams0, sc.pts0
    Q = Rotation.from_rotvec([0.3, -0.2, 0.5])
    s, tau = 1.7, np.array([0.4, -1.1, 0.25])
    pts2 = s * Q.apply(pts) + tau
    R = Rotation.from_rotvec(cams[:, :3])
    R2 = R * Q.inv()
    t2 = s * cams[:, 3:6] - R2.apply(np.broadcast_to(tau, (len(cams), 3)))
    cams2 = np.concatenate([R2.as_rotvec(), t2, cams[:, 6:]], axis=1)
    F1, _ = ob.cost(cams, pts)
    F2, _ = ob.cost(cams2, pts2)
    assert F2 == pytest.approx(F1, rel=1e-12)
    # depth priors break the scale part of the invariance
    sc_d = scenes.make_scene("small")
    ob_d = oracle.OracleBA.from_scene(sc_d)
    G1, _ = ob_d.cost(cams, pts)
    G2, _ = ob_d.cost(cams2, pts2)
    assert abs(G2 - G1) > 1e-6 * G1


def test_lm_accepted_costs_monotone_and_pcg_matches_direct():
    sc = scenes.make_scene("small")
    ob = oracle.OracleBA.from_scene(sc)
    _, _, rows_d = ob.lm(sc.cams0, sc.pts0, 10)
    ob.opts.solver = 1
    _, _, rows_p = ob.lm(sc.cams0, sc.pts0, 10)
    costs = [r["cost"] for r in rows_d]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    for a, b in zip(rows_d, rows_p):
        assert b["cost"] == pytest.approx(a["cost"], rel=1e-5)
        assert b["pcg_rel_res"] <= 1e-6


def test_residual_drop_is_sticky_and_thresholds_apply():
    sc = scenes.make_scene("small", scale=1.0)
    opts = oracle.OracleOptions(extract_every=2, drop_residual_px=4.0, min_cam_obs=15, min_pt_obs=2)
    ob = oracle.OracleBA.from_scene(sc, opts)
    alive = np.ones(sc.n_obs, np.uint8)
    c, p, rows = ob.lm(sc.cams0, sc.pts0, 5, alive=alive)
    dropped = alive == 0
    # outliers are uniform over the image: nearly all of them are dropped, few inliers are
    assert dropped[sc.is_outlier].mean() > 0.9
    assert dropped[~sc.is_outlier].mean() < 0.01
    assert rows[-1]["n_obs_act"] <= sc.n_obs - dropped.sum()


# --------------------------------------------------------------------------
# implicit adjoint (Sec. 3.3 normal equations at the optimum)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("w", [[0.0, 0.0, 0.0], [2e-5, -1e-5, 3e-5], [0.3, -0.7, 0.2],
                               [1.2, 2.1, -0.4], [0.0, 3.0, 0.1]])
def test_so3_left_jacobian_inverse_is_update_derivative(w):
    """d Log(Exp(dw) Exp(w)) / d dw at dw = 0, by central differences through SciPy."""
    w = np.asarray(w, dtype=np.float64)
    J = oracle.so3_left_jacobian_inv(w)
    h = 1e-6
    fd = np.zeros((3, 3))
    R = Rotation.from_rotvec(w)
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        wp = (Rotation.from_rotvec(e) * R).as_rotvec()
        wm = (Rotation.from_rotvec(-e) * R).as_rotvec()
        fd[:, j] = (wp - wm) / (2 * h)
    np.testing.assert_allclose(J, fd, atol=2e-8)


def _converge(ob, cams, pts, iters=40):
    c, p, _ = ob.lm(cams, pts, iters)
    return c, p


@pytest.mark.parametrize("model", [0, 1])
def test_adjoint_matches_finite_differences_of_reconverged_oracle(model):
    """Low-noise scene (0.01 px, depth-prior noise 1e-4, no outliers): Gauss-Newton
    is the exact Hessian up to O(residual), so the implicit gradient of L = |cams - gt|^2/2 + |pts - gt|^2/2
    with respect to pixels and depth priors matches central differences of the
    fully re-converged FP64 LM.  Both camera models; under the centre model (Sec.
    3.2) the k1, k2 slots are not parameters (held by a unit diagonal in the
    solve), so their loss gradient does not enter."""
    spec = dataclasses.replace(scenes.SPECS["small"], n_cams=6, n_pts=50, track_min=4,
                               track_max=4, track_mean=4, pixel_sigma=0.01, depth_sigma=1e-4,
                               seed=21)
    sc = scenes.make_scene(spec, outliers=False, camera_model="centre" if model else "radial")
    ob = oracle.OracleBA(sc.cams0.shape[0], sc.pts0.shape[0], sc.obs_cam, sc.obs_pt,
                         sc.obs_uv.copy(), sc.depth.copy(), sc.fixed_cams,
                         oracle.OracleOptions(camera_model=model))
    c, p = _converge(ob, sc.cams0, sc.pts0, 60)
    valid, _ = ob.predicate(c, p)
    ext = ob.extract(valid)
    assert ext["obs_mask"].all()

    def loss(cc, pp):
        return 0.5 * np.sum((cc - sc.cams_gt) ** 2) + 0.5 * np.sum((pp - sc.pts_gt) ** 2)

    duv, dd = ob.backward(c, p, ext, c - sc.cams_gt, p - sc.pts_gt)
    rng = np.random.default_rng(3)
    ks = rng.choice(sc.n_obs, 8, replace=False)
    kd = rng.choice(np.flatnonzero(sc.depth > 0), 4, replace=False)
    scale = max(np.abs(duv).max(), 1e-12)
    for k in ks:
        for j in range(2):
            h = 1e-4
            ob.obs_uv[k, j] += h
            Lp = loss(*_converge(ob, c, p))
            ob.obs_uv[k, j] -= 2 * h
            Lm = loss(*_converge(ob, c, p))
            ob.obs_uv[k, j] += h
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - duv[k, j]) <= 2e-3 * scale, (k, j, fd, duv[k, j])
    dscale = max(np.abs(dd).max(), 1e-12)
    for k in kd:
        h = 1e-3 * ob.depth[k]  # smaller steps move the cost by less than LM resolves
        ob.depth[k] += h
        Lp = loss(*_converge(ob, c, p))
        ob.depth[k] -= 2 * h
        Lm = loss(*_converge(ob, c, p))
        ob.depth[k] += h
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - dd[k]) <= 2e-3 * dscale, (k, fd, dd[k])
    # observations without a prior have no depth gradient
    assert np.all(dd[~(sc.depth > 0)] == 0.0)


# --------------------------------------------------------------------------
# LM control (Sec. 3.3): accept rule, damping schedule, reported RMSE
# --------------------------------------------------------------------------
# The paper names Marquardt damping but not its control; the reading is
# Nielsen's rule as given by Madsen, Nielsen & Tingleff, "Methods for non-linear
# least squares problems" (2004), Eq. 2.21 / Algorithm 3.16.  The expected values
# below were worked by hand from that rule and are written out as literals.

@pytest.mark.parametrize("lam, nu, accepted, gain, lam_new, nu_new", [
    (1e-4, 2.0, True, 0.5, 1e-4, 2.0),              # t = 0: factor 1
    (1e-4, 2.0, True, 0.75, 8.75e-5, 2.0),          # t = 0.5: 1 - 0.125
    (1e-4, 2.0, True, 0.25, 1.125e-4, 2.0),         # t = -0.5: 1 + 0.125
    (1e-4, 2.0, True, 0.9, 4.88e-5, 2.0),           # t = 0.8: 1 - 0.512
    (1e-4, 2.0, True, 0.002, 1.988047936e-4, 2.0),  # t = -0.996: 1 + 0.988047936
    (1e-4, 2.0, True, 1.0, 1e-4 / 3, 2.0),          # t = 1: 0, clamped to 1/3
    (3e-2, 2.0, True, 2.0, 1e-2, 2.0),              # t = 3: -26, clamped to 1/3
    (1e-4, 16.0, True, 0.5, 1e-4, 2.0),             # an accept resets nu
    (1e-4, 2.0, False, -5.0, 2e-4, 4.0),            # reject: lambda * nu, nu doubles
    (2e-4, 4.0, False, 1e-4, 8e-4, 8.0),
    (8e-4, 8.0, False, float("nan"), 6.4e-3, 16.0),
])
def test_damping_update_hand_worked(lam, nu, accepted, gain, lam_new, nu_new):
    got_l, got_n = oracle.lm_damping(accepted, gain, lam, nu)
    assert got_l == pytest.approx(lam_new, rel=1e-15)
    assert got_n == nu_new


@pytest.mark.parametrize("F, Fc, pred, expect", [
    (10.0, 9.0, 1.0, True),          # gain 1
    (10.0, 9.999, 1.0, False),       # gain 1e-3 exactly: not above the threshold
    (10.0, 9.9989, 1.0, True),       # gain 1.1e-3
    (10.0, 10.5, 1.0, False),        # cost went up
    (10.0, 9.0, 0.0, False),         # no predicted decrease
    (10.0, 9.0, -1.0, False),        # negative predicted decrease (gain -1 anyway)
    (10.0, 11.0, -1.0, False),       # both negative: gain +1, still rejected
    (10.0, float("nan"), 1.0, False),
    (10.0, float("inf"), 1.0, False),
])
def test_accept_rule_hand_worked(F, Fc, pred, expect):
    assert oracle.lm_accept(F, Fc, pred) == expect


def test_lm_trace_reject_chains_and_resets():
    """A start 30 degrees off with lambda0 = 1e-12 forces a chain of rejected steps.
    Fixed in advance: after an accepted step (or at the start) consecutive rejects
    multiply lambda by exactly 2, 4, 8, ...; an accepted step changes lambda by a
    factor in [1/3, 2), below 1 exactly when the gain exceeds 1/2, and exactly 1/3
    when the gain is at least (1 + (2/3)^(1/3)) / 2 = 0.93680; the accept decision
    is gain > 1e-3 with the gain recomputed from the logged costs."""
    spec = dataclasses.replace(scenes.SPECS["small"], n_cams=5, n_pts=40, track_min=3,
                               track_max=3, track_mean=3, seed=7, rot_perturb_deg=30.0)
    sc = scenes.make_scene(spec)
    ob = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(lambda0=1e-12))
    _, _, rows = ob.lm(sc.cams0, sc.pts0, 16)
    acc = [r["accepted"] for r in rows]
    assert sum(acc) >= 3 and len(acc) - sum(acc) >= 5, acc
    assert rows[0]["lam"] == 1e-12
    run = 0  # rejects since the last accept
    for prev, nxt in zip(rows, rows[1:]):
        gain = (prev["cost"] - prev["cand_cost"]) / prev["pred_decrease"]
        assert prev["accepted"] == (np.isfinite(gain) and prev["pred_decrease"] > 0 and gain > 1e-3)
        ratio = nxt["lam"] / prev["lam"]
        if prev["accepted"]:
            run = 0
            assert 1.0 / 3.0 * (1 - 1e-15) <= ratio < 2.0
            assert (ratio < 1.0) == (gain > 0.5)
            if gain >= 0.9368:
                assert ratio == pytest.approx(1.0 / 3.0, rel=1e-15)
        else:
            run += 1
            assert ratio == 2.0 ** run, (run, ratio)
        # a rejected step leaves the state, the active set and so the cost unchanged
        if not prev["accepted"]:
            assert nxt["cost"] == prev["cost"]
            assert nxt["n_obs_act"] == prev["n_obs_act"]


def test_rmse_and_cost_at_ground_truth_with_known_offsets():
    """At the true state with exact depth priors, every residual is a pixel offset
    that we place: RMSE = sqrt(mean |offset|^2) over the active observations and
    F = 1/2 sum rho(|offset|^2) with the Huber closed form, whatever the camera model."""
    spec = dataclasses.replace(scenes.SPECS["small"], n_cams=6, n_pts=60, track_min=4,
                               track_max=4, track_mean=4, seed=5)
    sc = scenes.make_scene(spec, noise=False, outliers=False)
    rng = np.random.default_rng(17)
    mags = rng.choice([0.3, 0.6, 0.9, 2.0, 5.0], size=sc.n_obs)
    ang = rng.uniform(0, 2 * math.pi, sc.n_obs)
    off = mags[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    mask = (rng.random(sc.n_obs) < 0.7).astype(np.uint8)
    for delta in (1.0, 0.0):
        ob = oracle.OracleBA(sc.cams0.shape[0], sc.pts0.shape[0], sc.obs_cam, sc.obs_pt,
                             sc.obs_uv + off, sc.depth, sc.fixed_cams,
                             oracle.OracleOptions(huber_delta=delta))
        for m in (None, mask):
            sel = np.ones(sc.n_obs, bool) if m is None else m.astype(bool)
            F, rmse = ob.cost(sc.cams_gt, sc.pts_gt, m)
            s = mags[sel]
            assert rmse == pytest.approx(math.sqrt(np.mean(s ** 2)), rel=1e-12)
            rho = np.where(s <= delta, s ** 2, 2 * delta * s - delta ** 2) if delta > 0 else s ** 2
            assert F == pytest.approx(0.5 * rho.sum(), rel=1e-11)


# --------------------------------------------------------------------------
# one-shot pruning vs dynamic extraction (Sec. 4.2)
# --------------------------------------------------------------------------

def test_one_shot_freezes_the_first_active_set_and_dynamic_readmits():
    """Injected frustum exits: points that start above the image of their nearer
    cameras.  One-shot pruning keeps the first iteration's active set for the whole
    run; per-iteration extraction (Sec. 4.2 step 3) re-admits the observations once
    the points come back into view, and ends with the smaller point error."""
    sc = scenes.make_scene("small", frustum_exit_frac=0.3)
    out = {}
    for mode in (0, 1):
        ob = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(extract_mode=mode))
        g0, _ = ob.predicate(sc.cams0, sc.pts0)
        c, p, rows = ob.lm(sc.cams0, sc.pts0, 12)
        acts = [r["n_obs_act"] for r in rows]
        assert acts[0] == int(g0.sum()) < sc.n_obs  # the injected exits are invalid at the start
        out[mode] = (acts, np.linalg.norm(p - sc.pts_gt, axis=1).mean())
    acts_once, err_once = out[1]
    acts_dyn, err_dyn = out[0]
    assert len(set(acts_once)) == 1
    gt_valid, _ = oracle.OracleBA.from_scene(sc).predicate(sc.cams_gt, sc.pts_gt)
    assert acts_dyn[-1] > acts_dyn[0] and acts_dyn[-1] >= int(gt_valid.sum()) - 10
    assert err_dyn < err_once


# --------------------------------------------------------------------------
# the camera parameterisation of Sec. 3.2 (centre, rotation, focal length)
# --------------------------------------------------------------------------

def test_centre_model_projection_closed_form_and_equivalence():
    """P = R (X - c): with R = I the pixel is f (X - c)_xy / (X - c)_z + (cx, cy); and
    the same camera as [w, t = -R c, f, 0, 0] under the radial model projects the
    same (one rotation, two parameterisations of its position)."""
    X = np.array([0.3, -0.2, 0.5])
    cam = np.array([0, 0, 0, 0.1, 0.05, -2.5, 480.0, 0.3, -0.2])  # k1, k2 ignored
    r, _, _, z, uvh = oracle.observe(cam, X, np.zeros(2), 0.0, 0.0, model=1)
    d = X - cam[3:6]
    assert z == pytest.approx(d[2], abs=1e-15)
    np.testing.assert_allclose(uvh, [480 * d[0] / d[2] + 320, 480 * d[1] / d[2] + 240], atol=1e-12)
    rng = np.random.default_rng(4)
    for _ in range(20):
        w = rng.normal(size=3) * 0.5
        c = rng.normal(size=3) + [0, 0, -3]
        R = Rotation.from_rotvec(w).as_matrix()
        X = rng.normal(size=3) * 0.3
        cam1 = np.concatenate([w, c, [500.0, 0.0, 0.0]])
        cam0 = np.concatenate([w, -R @ c, [500.0, 0.0, 0.0]])
        a = oracle.observe(cam1, X, [300.0, 200.0], 0.3, 1.0, model=1)
        b = oracle.observe(cam0, X, [300.0, 200.0], 0.3, 1.0, model=0)
        np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(a[2], b[2], rtol=1e-12, atol=1e-12)  # point block is the same


def test_centre_model_jacobian_central_fd():
    rng = np.random.default_rng(6)
    for trial in range(30):
        cam = np.concatenate([rng.normal(size=3) * 0.6, rng.normal(size=3) * 0.3 + [0, 0, -3],
                              [500 + 20 * rng.normal(), 0.1, -0.1]])
        X = rng.normal(size=3) * 0.5
        uv = rng.uniform(0, 600, 2)
        tau, wt = (1 / 3.1, 1.0) if trial % 2 else (0.0, 0.25)
        r0, Jc, Jp, _, _ = oracle.observe(cam, X, uv, tau, wt, model=1)
        h = 1e-6
        for i in range(9):
            rp = oracle.observe(_perturb_cam(cam, i, h), X, uv, tau, wt, model=1)[0]
            rm = oracle.observe(_perturb_cam(cam, i, -h), X, uv, tau, wt, model=1)[0]
            fd = (rp - rm) / (2 * h)
            np.testing.assert_allclose(Jc[:, i], fd, rtol=1e-7, atol=1e-7 * max(1.0, np.abs(fd).max()))
        assert not Jc[:, 7:].any()  # no distortion columns


def test_centre_model_step_vs_dense_and_noise_free_convergence():
    sc = tiny_scene(noise=True, outliers=True, camera_model="centre")
    opts = oracle.OracleOptions(camera_model=1, invalid_depth_weight=1e-3)
    ob = oracle.OracleBA.from_scene(sc, opts)
    cams, pts = sc.cams0, sc.pts0
    geom, _ = ob.predicate(cams, pts)
    ext = ob.extract(geom)
    ne = ob.normal_equations(cams, pts, ext["obs_mask"])
    H, g, free, act = _dense_system(ob, cams, pts, ext["obs_mask"], ext)
    lam = 1e-2
    dx = np.linalg.solve(H + lam * np.diag(np.clip(np.diag(H), 1e-6, 1e32)), -g)
    st = ob.solve_step(ne, ext, lam)
    got = np.concatenate([st["dc"][free].ravel(), st["dp"][act].ravel()])
    np.testing.assert_allclose(got, dx, rtol=1e-4, atol=1e-6 * np.abs(dx).max())
    assert not st["dc"][:, 7:].any()
    # exact measurements: the LM reaches zero cost and the true cameras
    sc0 = scenes.make_scene("small", noise=False, outliers=False, camera_model="centre")
    ob0 = oracle.OracleBA.from_scene(sc0, oracle.OracleOptions(camera_model=1))
    assert ob0.cost(sc0.cams_gt, sc0.pts_gt)[0] < 1e-18
    c, p, rows = ob0.lm(sc0.cams0, sc0.pts0, 20)
    assert ob0.cost(c, p)[0] <= 1e-20 * rows[0]["cost"]
    np.testing.assert_allclose(c[:, 3:7], sc0.cams_gt[:, 3:7], atol=1e-7)
