"""Implicit adjoint of the converged BA (ba_backward and the autograd op) against
the oracle's implicit gradient, and against central differences of re-converged
FP64 solves.  The loss is the squared error of the solution against ground
truth, L = |cams - cams_gt|^2 / 2 + |pts - pts_gt|^2 / 2."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2510_13310_b300 import ba, scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

SOLVERS = [ba.BA_SOLVER_EXPLICIT, ba.BA_SOLVER_IMPLICIT]


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def oracle_gradient(sc, cams, pts):
    orc = oracle.OracleBA.from_scene(sc)
    geom, _ = orc.predicate(cams, pts)
    ext = orc.extract(geom)
    duv, dd = orc.backward(cams, pts, ext, cams - sc.cams_gt, pts - sc.pts_gt)
    return duv, dd, ext


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("precision,tol", [(ba.BA_FP64, 1e-6), (ba.BA_FP32, 2e-2)])
def test_backward_matches_oracle_on_differentiable_workload(precision, tol, solver):
    """The differentiable-BA workload: 100 cameras, 20k points, ~200k observations."""
    sc = scenes.make_scene("diff")
    fp64 = precision == ba.BA_FP64
    gpu = ba.Problem.from_scene(sc, ba.Options(precision=precision, solver=solver,
                                               pcg_rel_tol=1e-11 if fp64 else 1e-6))
    gpu.solve(10)
    cams, pts = gpu.get_params()
    duv_g, dd_g = gpu.backward(cams - sc.cams_gt, pts - sc.pts_gt)
    duv_o, dd_o, ext = oracle_gradient(sc, cams, pts)
    om = gpu.get_active()["obs_mask"]
    assert np.array_equal(om, ext["obs_mask"])
    e_uv, e_d = rel_err(duv_g, duv_o), rel_err(dd_g, dd_o)
    print(f"ba_backward vs oracle implicit gradient: uv {e_uv:.3e}, depth {e_d:.3e}")
    assert e_uv < tol
    assert e_d < tol
    # inactive observations and those without a prior carry no gradient
    assert not duv_g[om == 0].any()
    assert not dd_g[~(sc.depth > 0)].any()
    gpu.close()


def low_noise_scene():
    # pixel noise 0.01 px and depth-prior noise 1e-4 (relative), no outliers: the
    # residuals are small enough that Gauss-Newton is the exact Hessian to ~1e-4
    spec = dataclasses.replace(scenes.SPECS["small"], n_cams=8, n_pts=300, track_min=4, track_max=6,
                               track_mean=5, pixel_sigma=0.01, depth_sigma=1e-4, seed=31)
    return scenes.make_scene(spec, outliers=False)


def solve_from(sc, cams, pts, uv, depth, opts, iters=40):
    p = ba.Problem(cams, pts, sc.obs_cam, sc.obs_pt, uv, depth, opts)
    p.solve(iters)
    c, q = p.get_params()
    p.close()
    return c, q


def test_fp64_backward_matches_reconverged_finite_differences():
    sc = low_noise_scene()
    opts = ba.Options(precision=ba.BA_FP64, pcg_rel_tol=1e-12, fixed_cams=tuple(sc.fixed_cams))
    c, p = solve_from(sc, sc.cams0, sc.pts0, sc.obs_uv, sc.depth, opts, 60)
    gpu = ba.Problem(c, p, sc.obs_cam, sc.obs_pt, sc.obs_uv, sc.depth, opts)
    duv, dd = gpu.backward(c - sc.cams_gt, p - sc.pts_gt)
    gpu.close()

    def loss(cc, pp):
        return 0.5 * np.sum((cc - sc.cams_gt) ** 2) + 0.5 * np.sum((pp - sc.pts_gt) ** 2)

    rng = np.random.default_rng(5)
    scale = np.abs(duv).max()
    for k in rng.choice(sc.n_obs, 10, replace=False):
        for j in range(2):
            # the re-converged LM stops at rounding-level cost differences; the quotient
            # divides that noise by h, so h = 3e-4 px (truncation error O(h^2) negligible)
            h = 3e-4
            uv = sc.obs_uv.copy()
            uv[k, j] += h
            Lp = loss(*solve_from(sc, c, p, uv, sc.depth, opts))
            uv[k, j] -= 2 * h
            Lm = loss(*solve_from(sc, c, p, uv, sc.depth, opts))
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - duv[k, j]) <= 2e-3 * scale, (k, j, fd, duv[k, j])
    dscale = np.abs(dd).max()
    for k in rng.choice(np.flatnonzero(sc.depth > 0), 5, replace=False):
        h = 1e-3 * sc.depth[k]
        d = sc.depth.copy()
        d[k] += h
        Lp = loss(*solve_from(sc, c, p, sc.obs_uv, d, opts))
        d[k] -= 2 * h
        Lm = loss(*solve_from(sc, c, p, sc.obs_uv, d, opts))
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - dd[k]) <= 2e-3 * dscale, (k, fd, dd[k])


# FP32: the depth priors constrain the scale direction about 1e-6 as stiffly as
# the pixels constrain the rest ((1/z^2)^2 against (f/z)^2 per observation), so
# FP32 arithmetic resolves that component of mu, which the depth gradients
# mostly see, to a few percent; pixel gradients are accurate to ~1e-3.
@pytest.mark.parametrize("precision,tol_uv,tol_d", [(ba.BA_FP64, 1e-7, 1e-7), (ba.BA_FP32, 1e-2, 1.5e-1)])
def test_autograd_op_gives_the_implicit_gradient(precision, tol_uv, tol_d):
    sc = low_noise_scene()
    dev = torch.device("cuda")
    t = lambda a, **kw: torch.tensor(a, device=dev, **kw)
    uv = t(sc.obs_uv, dtype=torch.float64, requires_grad=True)
    depth = t(sc.depth, dtype=torch.float64, requires_grad=True)
    opts = ba.Options(precision=precision, pcg_rel_tol=1e-12 if precision == ba.BA_FP64 else 1e-6,
                      fixed_cams=tuple(sc.fixed_cams))
    cams, pts = ba.bundle_adjust(t(sc.cams0), t(sc.pts0), uv, depth, t(sc.obs_cam), t(sc.obs_pt),
                                 options=opts, iters=30)
    loss = 0.5 * ((cams - t(sc.cams_gt)) ** 2).sum() + 0.5 * ((pts - t(sc.pts_gt)) ** 2).sum()
    loss.backward()
    c, p = cams.detach().cpu().numpy(), pts.detach().cpu().numpy()
    duv_o, dd_o, _ = oracle_gradient(sc, c, p)
    e_uv = rel_err(uv.grad.cpu().numpy(), duv_o)
    e_d = rel_err(depth.grad.cpu().numpy(), dd_o)
    print(f"autograd vs oracle implicit gradient: uv {e_uv:.3e}, depth {e_d:.3e}")
    assert e_uv < tol_uv
    assert e_d < tol_d
