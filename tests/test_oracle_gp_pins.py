"""Pins of the FP64 global-positioning oracle (Sec. 3.1 Eq. GP objective, Sec. 4.1
depth-constrained GP, Sec. 3.3 Eq. LM) against routes independent of it: central
finite differences, a dense NumPy solve of the full damped system (free centres,
points and free scales together), NumPy set membership, exact convergence and
the objective's invariances."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2510_13310_b300 import scenes


def tiny_gp(n_cams=5, n_pts=30, track=3, seed=7, **kw):
    spec = dataclasses.replace(scenes.SPECS["small"], n_cams=n_cams, n_pts=n_pts, track_min=track,
                               track_max=track, track_mean=track, seed=seed)
    return scenes.make_gp_scene(spec, **kw)


def test_gp_residual_jacobians_central_fd():
    rng = np.random.default_rng(3)
    for _ in range(20):
        t, X = rng.normal(size=3), rng.normal(size=3)
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        s = rng.uniform(0.2, 2.0)
        u, Jt, JX, Js = oracle.gp_residual(t, X, v, s)
        np.testing.assert_allclose(u, v - s * (X - t), rtol=1e-15, atol=1e-15)
        h = 1e-6
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            fd_t = (oracle.gp_residual(t + e, X, v, s)[0] - oracle.gp_residual(t - e, X, v, s)[0]) / (2 * h)
            fd_x = (oracle.gp_residual(t, X + e, v, s)[0] - oracle.gp_residual(t, X - e, v, s)[0]) / (2 * h)
            np.testing.assert_allclose(Jt[:, i], fd_t, atol=1e-8)
            np.testing.assert_allclose(JX[:, i], fd_x, atol=1e-8)
        fd_s = (oracle.gp_residual(t, X, v, s + h)[0] - oracle.gp_residual(t, X, v, s - h)[0]) / (2 * h)
        np.testing.assert_allclose(Js, fd_s, atol=1e-8)


def test_gp_free_set_is_set_membership():
    """Sec. 4.1: S_free = {k | m_k = 0}, compacted by rank; NaN and non-positive
    depths count as missing."""
    sc = tiny_gp(n_cams=8, n_pts=60, track=4)
    depth = sc.depth.copy()
    depth[::7] = np.nan
    depth[3::11] = -1.0
    og = oracle.OracleGP(sc.centres0.shape[0], sc.pts0.shape[0], sc.obs_cam, sc.obs_pt, sc.rays, depth)
    fr, n = og.free_set()
    free = ~(np.nan_to_num(depth, nan=-1.0) > 0)
    idx = np.flatnonzero(free)
    assert n == idx.size
    exp = np.full(sc.n_obs, -1)
    exp[idx] = np.searchsorted(idx, idx)
    np.testing.assert_array_equal(fr, exp)


def _dense_gp_system(og, t, X, s, delta):
    """Dense robust-weighted J^T J and J^T u over (free centres, points, free
    scales), J from central differences of the residual."""
    C, P, N = og.n_cams, og.n_pts, og.n_obs
    free_c = [c for c in range(C) if not og.fixed[c] and (og.obs_cam == c).any()]
    fr, _ = og.free_set()
    free_k = [k for k in range(N) if fr[k] >= 0]
    cols = [("t", c, i) for c in free_c for i in range(3)] + [("X", p, i) for p in range(P) for i in range(3)] \
        + [("s", k, 0) for k in free_k]

    def resid(tt, XX, ss):
        sc_ = np.where(og.depth > 0, 1.0 / np.where(og.depth > 0, og.depth, 1.0), ss)
        return og.rays - sc_[:, None] * (XX[og.obs_pt] - tt[og.obs_cam])

    base = resid(t, X, s)
    n2 = (base ** 2).sum(1)
    w = np.where(n2 <= delta ** 2, 1.0, delta / np.sqrt(n2)) if delta > 0 else np.ones(N)
    J = np.zeros((N, 3, len(cols)))
    h = 1e-7
    for j, (kind, idx, i) in enumerate(cols):
        tp, tm, Xp, Xm, sp, sm = t.copy(), t.copy(), X.copy(), X.copy(), s.copy(), s.copy()
        if kind == "t":
            tp[idx, i] += h
            tm[idx, i] -= h
        elif kind == "X":
            Xp[idx, i] += h
            Xm[idx, i] -= h
        else:
            sp[idx] += h
            sm[idx] -= h
        J[:, :, j] = (resid(tp, Xp, sp) - resid(tm, Xm, sm)) / (2 * h)
    H = np.einsum("k,kai,kaj->ij", w, J, J)
    g = np.einsum("k,kai,ka->i", w, J, base)
    return H, g, free_c, free_k


@pytest.mark.parametrize("delta", [0.1, 0.0])
def test_gp_damped_step_vs_dense_full_system(delta):
    sc = tiny_gp(noise=True, outliers=True)
    og = oracle.OracleGP.from_scene(sc, oracle.OracleGPOptions(huber_delta=delta))
    t, X, s = sc.centres0, sc.pts0, sc.scales0
    H, g, free_c, free_k = _dense_gp_system(og, t, X, s, delta)
    for lam in (1e-2, 1e-5):
        D = np.clip(np.diag(H), 1e-6, 1e32)
        dx = np.linalg.solve(H + lam * np.diag(D), -g)
        st = og.solve_step(t, X, s, lam)
        assert st["status"] == 0
        got = np.concatenate([st["dt"][free_c].ravel(), st["dX"].ravel(), st["ds"][free_k]])
        np.testing.assert_allclose(got, dx, rtol=1e-5, atol=1e-7 * np.abs(dx).max())
        pred = -g @ dx - 0.5 * dx @ H @ dx
        assert st["pred_decrease"] == pytest.approx(pred, rel=1e-6)
        assert not st["dt"][sc.fixed_cams].any()
        assert not st["ds"][sc.depth > 0].any()


@pytest.mark.parametrize("depth_frac", [0.5, 0.05])
def test_gp_noise_free_converges_to_truth(depth_frac):
    """Exact rays: the LM reaches zero cost, and the pinned scales (s = 1/d) fix the
    metric scale, so centres and points land on the truth (camera 0 fixes translation)."""
    spec = dataclasses.replace(scenes.SPECS["small"], depth_frac=depth_frac)
    sc = scenes.make_gp_scene(spec, noise=False, outliers=False)
    og = oracle.OracleGP.from_scene(sc)
    t, X, s, rows = og.lm(sc.centres0, sc.pts0, sc.scales0, 20)
    F, _ = og.cost(t, X, s)
    assert F <= 1e-20 * rows[0]["cost"]
    np.testing.assert_allclose(t, sc.centres_gt, atol=1e-9)
    np.testing.assert_allclose(X, sc.pts_gt, atol=1e-9)
    acc = [r["cost"] for r in rows if r["accepted"]]
    assert all(b <= a for a, b in zip(acc, acc[1:]))


def test_gp_cost_invariances():
    """The GP objective is invariant to a common translation of centres and points;
    without depth priors also to a common scale alpha (t, X -> alpha t, alpha X,
    s -> s / alpha); pinned scales break the latter (they carry metric scale)."""
    sc = tiny_gp(n_cams=6, n_pts=40, track=4, seed=2)
    tau, alpha = np.array([0.3, -1.2, 0.7]), 1.9
    og_free = oracle.OracleGP(sc.centres0.shape[0], sc.pts0.shape[0], sc.obs_cam, sc.obs_pt, sc.rays,
                              np.zeros(sc.n_obs))
    F0, _ = og_free.cost(sc.centres0, sc.pts0, sc.scales0)
    F1, _ = og_free.cost(sc.centres0 + tau, sc.pts0 + tau, sc.scales0)
    F2, _ = og_free.cost(alpha * sc.centres0, alpha * sc.pts0, sc.scales0 / alpha)
    assert F1 == pytest.approx(F0, rel=1e-12) and F2 == pytest.approx(F0, rel=1e-12)
    og = oracle.OracleGP.from_scene(sc)
    G0, _ = og.cost(sc.centres0, sc.pts0, sc.scales0)
    G1, _ = og.cost(sc.centres0 + tau, sc.pts0 + tau, sc.scales0)
    G2, _ = og.cost(alpha * sc.centres0, alpha * sc.pts0, sc.scales0 / alpha)
    assert G1 == pytest.approx(G0, rel=1e-12)
    assert abs(G2 - G0) > 1e-3 * G0


def test_gp_huber_closed_form():
    """One observation with a chosen residual: F = 1/2 rho(|u|^2) with Huber's closed form."""
    for du, delta, expect in [(0.05, 0.1, 0.0025), (0.3, 0.1, 2 * 0.1 * 0.3 - 0.01), (0.3, 0.0, 0.09)]:
        og = oracle.OracleGP(1, 1, [0], [0], [[1.0, 0.0, 0.0]], [0.0], fixed_cams=[],
                             opts=oracle.OracleGPOptions(huber_delta=delta))
        # X - t = (1 - du, 0, 0) with s = 1: u = (du, 0, 0)
        F, rms = og.cost([[0.0, 0.0, 0.0]], [[1.0 - du, 0.0, 0.0]], [1.0])
        assert F == pytest.approx(0.5 * expect, rel=1e-12)
        assert rms == pytest.approx(du, rel=1e-12)
