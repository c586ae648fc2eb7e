"""Element-wise comparison helpers for the GPU parity tests.

Every comparison is per element: |got - ref| <= atol_e + rtol |ref|, where the
absolute part atol_e is the tolerance times a scale that the mathematics gives
for that element (never the largest entry of the whole array):
  - a symmetric positive semi-definite block A (U_c, V_p): |A_ij| <= sqrt(A_ii A_jj)
    (Cauchy-Schwarz), so the scale of entry (i, j) is sqrt(|A_ii| |A_jj|);
  - a gradient g = sum_k rho'_k J_k^T r_k: |g_i| <= sqrt(H_ii) sqrt(sum_k rho'_k |r_k|^2),
    with the sum over the observations of that camera or point;
  - a coupling block W_k = rho'_k J_c^T J_p: |W_ij| <= rho'_k |J_c[:, i]| |J_p[:, j]|;
  - a solution vector (a damped step, a gradient): per parameter kind, the
    largest magnitude of that kind (rotation, translation, focal, k1, k2 and
    point coordinates have different units).
"""
from __future__ import annotations

import numpy as np
import pytest


def check_close(got, ref, rtol, atol=0.0, label=""):
    """Assert |got - ref| <= atol + rtol |ref| element-wise (atol broadcastable).
    Returns the worst ratio |got - ref| / (atol + rtol |ref|)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (label, got.shape, ref.shape)
    bound = np.broadcast_to(np.asarray(atol, dtype=np.float64), ref.shape) + rtol * np.abs(ref)
    err = np.abs(got - ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), np.where(err > 0, np.inf, 0.0))
    worst = float(ratio.max()) if ratio.size else 0.0
    if not np.all(np.isfinite(got)) or worst > 1.0:
        i = np.unravel_index(int(np.argmax(ratio)), ratio.shape) if ratio.size else ()
        raise AssertionError(f"{label}: worst element {i}: got {got[i]!r}, ref {ref[i]!r}, "
                             f"bound {bound[i]!r} (ratio {worst:.3g})")
    return worst


def sym_scale(blocks):
    """sqrt(|A_ii| |A_jj|) for a stack of square blocks [..., n, n]."""
    d = np.sqrt(np.abs(np.einsum("...ii->...i", blocks)))
    return d[..., :, None] * d[..., None, :]


def kind_scale(x):
    """Per-column largest magnitude of [rows, m] (one column per parameter kind)."""
    x = np.asarray(x, dtype=np.float64)
    return np.abs(x).max(axis=0, keepdims=True) if x.size else np.zeros((1,) + x.shape[1:])


def robust_weights(r, delta):
    """Huber IRLS weights rho'(s) = min(1, delta / sqrt(s)) of stacked residuals r [N, 3]."""
    s = (np.asarray(r) ** 2).sum(1)
    if delta <= 0:
        return np.ones_like(s)
    return np.where(s <= delta * delta, 1.0, delta / np.sqrt(np.maximum(s, 1e-300)))


def normal_equation_scales(orc, cams, pts, obs_mask):
    """Per-element scales of U, V, g_c, g_p and W (see the module docstring) at a
    state, from the oracle's per-observation residuals and Jacobians."""
    ev = orc.eval_obs(cams, pts, want_jac=True)
    m = np.asarray(obs_mask, dtype=bool)
    w = robust_weights(ev["r"], orc.opts.huber_delta) * m
    rr = w * (ev["r"] ** 2).sum(1)
    C, P = orc.n_cams, orc.n_pts
    res_c = np.bincount(orc.obs_cam, weights=rr, minlength=C)
    res_p = np.bincount(orc.obs_pt, weights=rr, minlength=P)
    jc = np.sqrt((ev["Jc"] ** 2).sum(1))  # [N, 9] column norms
    jp = np.sqrt((ev["Jp"] ** 2).sum(1))  # [N, 3]
    w_scale = w[:, None, None] * jc[:, :, None] * jp[:, None, :]
    return dict(res_c=res_c, res_p=res_p, W=w_scale)


def check_blocks(lin, ne, orc, cams, pts, obs_mask, live, tol, W_rows=None):
    """Element-wise bars on the normal-equation blocks: every entry within tol of
    its Cauchy-Schwarz scale (sqrt(A_ii A_jj) for U and V; sqrt(H_ii) times the
    root of the weighted squared residuals for the gradients; rho' |J_c,i| |J_p,j|
    for W) plus tol relative."""
    s = normal_equation_scales(orc, cams, pts, obs_mask)
    dU = np.sqrt(np.abs(np.einsum("cii->ci", ne["U"])))
    dV = np.sqrt(np.abs(np.einsum("pii->pi", ne["V"])))
    worst = dict(U=check_close(lin["U"][live], ne["U"][live], tol, tol * sym_scale(ne["U"][live]), "U"),
                 V=check_close(lin["V"], ne["V"], tol, tol * sym_scale(ne["V"]), "V"),
                 gc=check_close(lin["gc"][live], ne["gc"][live], tol,
                                tol * (dU * np.sqrt(s["res_c"])[:, None])[live], "gc"),
                 gp=check_close(lin["gp"], ne["gp"], tol, tol * dV * np.sqrt(s["res_p"])[:, None], "gp"))
    rows = slice(None) if W_rows is None else W_rows
    worst["W"] = check_close(lin["W"][rows], ne["W"][rows], tol, tol * s["W"][rows], "W")
    return worst


def check_step(g, o, tol, pred_tol):
    """Damped steps element-wise: within tol of each parameter kind's scale (the
    largest magnitude of that camera parameter, or of the point coordinates) plus
    tol relative; the predicted decrease within pred_tol relative."""
    check_close(g["dc"], o["dc"], tol, tol * kind_scale(o["dc"]), "dc")
    check_close(g["dp"], o["dp"], tol, tol * kind_scale(o["dp"]), "dp")
    assert g["pred_decrease"] == pytest.approx(o["pred_decrease"], rel=pred_tol)
