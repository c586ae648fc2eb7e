"""ctypes wrapper of the FP64 CPU oracles (oracle/ba_oracle.c: bundle adjustment;
oracle/gp_oracle.c: depth-constrained global positioning).

TEST INFRASTRUCTURE ONLY.  The oracle is what the CUDA path is checked against;
only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
Every function here is argument marshalling; the arithmetic is in ba_oracle.c,
whose header cites the paper's section and equation for each step.
"""
from __future__ import annotations

import ctypes as ct
import dataclasses

import numpy as np

from . import build as _build

_LIB = None

c_i64 = ct.c_int64
P_f64 = ct.POINTER(ct.c_double)
P_i32 = ct.POINTER(ct.c_int32)
P_u8 = ct.POINTER(ct.c_uint8)


class Problem(ct.Structure):
    _fields_ = [("n_cams", c_i64), ("n_pts", c_i64), ("n_obs", c_i64),
                ("obs_cam", P_i32), ("obs_pt", P_i32), ("obs_uv", P_f64),
                ("depth", P_f64), ("fixed", P_u8)]


class Opts(ct.Structure):
    _fields_ = [("img_w", ct.c_int), ("img_h", ct.c_int), ("cx", ct.c_double), ("cy", ct.c_double),
                ("huber_delta", ct.c_double), ("depth_weight", ct.c_double),
                ("invalid_depth_weight", ct.c_double), ("min_depth", ct.c_double),
                ("extract_every", ct.c_int), ("drop_residual_px", ct.c_double),
                ("min_cam_obs", ct.c_int), ("min_pt_obs", ct.c_int), ("lambda0", ct.c_double),
                ("pcg_rel_tol", ct.c_double), ("pcg_max_iters", ct.c_int), ("solver", ct.c_int),
                ("extract_mode", ct.c_int), ("nu0", ct.c_double), ("camera_model", ct.c_int)]


class GPProblem(ct.Structure):
    _fields_ = [("n_cams", c_i64), ("n_pts", c_i64), ("n_obs", c_i64),
                ("obs_cam", P_i32), ("obs_pt", P_i32), ("rays", P_f64),
                ("depth", P_f64), ("fixed", P_u8)]


class GPOpts(ct.Structure):
    _fields_ = [("huber_delta", ct.c_double), ("lambda0", ct.c_double)]


class IterLog(ct.Structure):
    _fields_ = [("cost", ct.c_double), ("rmse_px", ct.c_double), ("lambda_", ct.c_double),
                ("gain", ct.c_double), ("pred_decrease", ct.c_double), ("cand_cost", ct.c_double),
                ("accepted", ct.c_int), ("pcg_iters", ct.c_int), ("pcg_rel_res", ct.c_double),
                ("n_cam_act", c_i64), ("n_pt_act", c_i64), ("n_obs_act", c_i64)]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ct.CDLL(path)
        L.oracle_default_opts.argtypes = [ct.POINTER(Opts)]
        L.oracle_rotvec_to_matrix.argtypes = [P_f64, P_f64]
        L.oracle_rotvec_compose.argtypes = [P_f64, P_f64, P_f64]
        L.oracle_so3_left_jacobian_inv.argtypes = [P_f64, P_f64]
        L.oracle_observe.argtypes = [P_f64, P_f64, P_f64, ct.c_double, ct.c_double, ct.c_double,
                                     ct.c_double, P_f64, P_f64, P_f64, P_f64, P_f64]
        L.oracle_observe_model.argtypes = [ct.c_int, P_f64, P_f64, P_f64, ct.c_double, ct.c_double,
                                           ct.c_double, ct.c_double, P_f64, P_f64, P_f64, P_f64, P_f64]
        L.oracle_eval_obs.argtypes = [ct.POINTER(Problem), ct.POINTER(Opts), P_f64, P_f64, P_f64,
                                      P_f64, P_f64, P_f64, P_f64]
        L.oracle_cost.argtypes = [ct.POINTER(Problem), ct.POINTER(Opts), P_f64, P_f64, P_u8, P_f64]
        L.oracle_cost.restype = ct.c_double
        L.oracle_predicate.argtypes = [ct.POINTER(Problem), ct.POINTER(Opts), P_f64, P_f64, P_u8, P_f64]
        L.oracle_extract.argtypes = [ct.POINTER(Problem), ct.POINTER(Opts), P_u8, P_u8, P_u8, P_u8,
                                     P_i32, P_i32, ct.POINTER(c_i64), ct.POINTER(c_i64)]
        L.oracle_extract.restype = ct.c_int
        L.oracle_normal_equations.argtypes = [ct.POINTER(Problem), ct.POINTER(Opts), P_f64, P_f64,
                                              P_u8, P_f64, P_f64, P_f64, P_f64, P_f64]
        L.oracle_schur_dense.argtypes = [ct.POINTER(Problem), P_f64, P_f64, P_f64, P_f64, P_f64,
                                         P_u8, P_i32, P_i32, c_i64, ct.c_double, P_f64, P_f64]
        L.oracle_solve_step.argtypes = [ct.POINTER(Problem), ct.POINTER(Opts), P_f64, P_f64, P_f64,
                                        P_f64, P_f64, P_u8, P_i32, P_i32, c_i64, ct.c_double,
                                        P_f64, P_f64, P_f64, P_f64]
        L.oracle_solve_step.restype = ct.c_int
        L.oracle_apply_step.argtypes = [c_i64, c_i64, P_f64, P_f64, P_f64, P_f64, P_f64, P_f64]
        L.oracle_lm.argtypes = [ct.POINTER(Problem), ct.POINTER(Opts), ct.c_int, P_f64, P_f64,
                                ct.POINTER(IterLog), P_u8]
        L.oracle_lm.restype = ct.c_int
        L.oracle_backward.argtypes = [ct.POINTER(Problem), ct.POINTER(Opts), P_f64, P_f64, P_u8,
                                      P_i32, P_i32, c_i64, P_f64, P_f64, P_f64, P_f64]
        L.oracle_backward.restype = ct.c_int
        L.oracle_lm_accept.argtypes = [ct.c_double, ct.c_double, ct.c_double]
        L.oracle_lm_accept.restype = ct.c_int
        L.oracle_lm_damping.argtypes = [ct.c_int, ct.c_double, ct.POINTER(ct.c_double),
                                        ct.POINTER(ct.c_double)]
        GP = ct.POINTER(GPProblem)
        GO = ct.POINTER(GPOpts)
        L.oracle_gp_residual.argtypes = [P_f64, P_f64, P_f64, ct.c_double, P_f64, P_f64, P_f64, P_f64]
        L.oracle_gp_free_set.argtypes = [GP, P_i32]
        L.oracle_gp_free_set.restype = c_i64
        L.oracle_gp_cost.argtypes = [GP, GO, P_f64, P_f64, P_f64, P_f64]
        L.oracle_gp_cost.restype = ct.c_double
        L.oracle_gp_normal_equations.argtypes = [GP, GO, P_f64, P_f64, P_f64] + [P_f64] * 9
        L.oracle_gp_solve_step.argtypes = [GP, GO, P_f64, P_f64, P_f64, ct.c_double, P_f64, P_f64,
                                           P_f64, P_f64]
        L.oracle_gp_solve_step.restype = ct.c_int
        L.oracle_gp_lm.argtypes = [GP, GO, ct.c_int, P_f64, P_f64, P_f64, ct.POINTER(IterLog)]
        L.oracle_gp_lm.restype = ct.c_int
        L.oracle_set_threads.argtypes = [ct.c_int]
        L.oracle_get_threads.restype = ct.c_int
        _LIB = L
    return _LIB


def _p(a, ptype):
    return a.ctypes.data_as(ptype)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclasses.dataclass
class OracleOptions:
    img_w: int = 640
    img_h: int = 480
    cx: float = 320.0
    cy: float = 240.0
    huber_delta: float = 1.0
    depth_weight: float = 1.0
    invalid_depth_weight: float = 0.0
    min_depth: float = 0.1
    extract_every: int = 0
    drop_residual_px: float = 0.0
    min_cam_obs: int = 1
    min_pt_obs: int = 1
    lambda0: float = 1e-4
    pcg_rel_tol: float = 1e-6
    pcg_max_iters: int = 500
    solver: int = 0  # 0 dense Cholesky of the Schur system, 1 PCG
    extract_mode: int = 0  # 0 dynamic (every iteration), 1 one-shot at the first iteration
    nu0: float = 2.0  # initial damping growth factor (a restart after rejected steps)
    camera_model: int = 0  # 0 radial [w, t, f, k1, k2]; 1 centre + rotation + focal [w, c, f, -, -]

    def to_c(self) -> Opts:
        return Opts(**dataclasses.asdict(self))


class OracleBA:
    """Holds one problem's arrays (host, input order) for repeated oracle calls."""

    def __init__(self, n_cams, n_pts, obs_cam, obs_pt, obs_uv, depth, fixed_cams=(0,),
                 opts: OracleOptions | None = None):
        self.L = lib()
        self.n_cams, self.n_pts = int(n_cams), int(n_pts)
        self.obs_cam = np.ascontiguousarray(obs_cam, dtype=np.int32)
        self.obs_pt = np.ascontiguousarray(obs_pt, dtype=np.int32)
        self.obs_uv = _f64(obs_uv).reshape(-1, 2)
        self.depth = _f64(depth)
        self.fixed = np.zeros(self.n_cams, dtype=np.uint8)
        self.fixed[np.asarray(fixed_cams, dtype=np.int64)] = 1
        self.n_obs = int(self.obs_cam.shape[0])
        self.opts = opts or OracleOptions()
        self._pb = Problem(self.n_cams, self.n_pts, self.n_obs, _p(self.obs_cam, P_i32),
                           _p(self.obs_pt, P_i32), _p(self.obs_uv, P_f64), _p(self.depth, P_f64),
                           _p(self.fixed, P_u8))

    @classmethod
    def from_scene(cls, scene, opts: OracleOptions | None = None):
        return cls(scene.cams0.shape[0], scene.pts0.shape[0], scene.obs_cam, scene.obs_pt,
                   scene.obs_uv, scene.depth, scene.fixed_cams, opts)

    def _o(self):
        return ct.byref(self.opts.to_c())

    # --- per-observation model ------------------------------------------------
    def eval_obs(self, cams, pts, want_jac=True):
        cams, pts = _f64(cams), _f64(pts)
        N = self.n_obs
        r = np.zeros((N, 3))
        z = np.zeros(N)
        uvh = np.zeros((N, 2))
        Jc = np.zeros((N, 3, 9)) if want_jac else None
        Jp = np.zeros((N, 3, 3)) if want_jac else None
        self.L.oracle_eval_obs(ct.byref(self._pb), self._o(), _p(cams, P_f64), _p(pts, P_f64),
                               _p(r, P_f64), _p(Jc, P_f64) if want_jac else None,
                               _p(Jp, P_f64) if want_jac else None, _p(z, P_f64), _p(uvh, P_f64))
        return dict(r=r, Jc=Jc, Jp=Jp, z=z, uvhat=uvh)

    def cost(self, cams, pts, mask=None):
        rm = ct.c_double(0)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        F = self.L.oracle_cost(ct.byref(self._pb), self._o(), _p(_f64(cams), P_f64),
                               _p(_f64(pts), P_f64), None if m is None else _p(m, P_u8), ct.byref(rm))
        return F, rm.value

    def predicate(self, cams, pts):
        g = np.zeros(self.n_obs, dtype=np.uint8)
        res = np.zeros(self.n_obs)
        self.L.oracle_predicate(ct.byref(self._pb), self._o(), _p(_f64(cams), P_f64),
                                _p(_f64(pts), P_f64), _p(g, P_u8), _p(res, P_f64))
        return g, res

    def extract(self, valid):
        valid = np.ascontiguousarray(valid, dtype=np.uint8)
        cm = np.zeros(self.n_cams, np.uint8)
        pm = np.zeros(self.n_pts, np.uint8)
        om = np.zeros(self.n_obs, np.uint8)
        cr = np.zeros(self.n_cams, np.int32)
        pr = np.zeros(self.n_pts, np.int32)
        ncf, npa = c_i64(0), c_i64(0)
        rounds = self.L.oracle_extract(ct.byref(self._pb), self._o(), _p(valid, P_u8), _p(cm, P_u8),
                                       _p(pm, P_u8), _p(om, P_u8), _p(cr, P_i32), _p(pr, P_i32),
                                       ct.byref(ncf), ct.byref(npa))
        return dict(cam_mask=cm, pt_mask=pm, obs_mask=om, cam_rank=cr, pt_rank=pr,
                    n_cam_free=ncf.value, n_pt_act=npa.value, rounds=rounds)

    def normal_equations(self, cams, pts, obs_mask):
        C, P, N = self.n_cams, self.n_pts, self.n_obs
        U = np.zeros((C, 9, 9)); V = np.zeros((P, 3, 3)); W = np.zeros((N, 9, 3))
        gc = np.zeros((C, 9)); gp = np.zeros((P, 3))
        om = np.ascontiguousarray(obs_mask, dtype=np.uint8)
        self.L.oracle_normal_equations(ct.byref(self._pb), self._o(), _p(_f64(cams), P_f64),
                                       _p(_f64(pts), P_f64), _p(om, P_u8), _p(U, P_f64), _p(V, P_f64),
                                       _p(W, P_f64), _p(gc, P_f64), _p(gp, P_f64))
        return dict(U=U, V=V, W=W, gc=gc, gp=gp)

    def schur_dense(self, ne, ext, lam):
        n = 9 * ext["n_cam_free"]
        S = np.zeros((n, n)); b = np.zeros(n)
        self.L.oracle_schur_dense(ct.byref(self._pb), _p(ne["U"], P_f64), _p(ne["V"], P_f64),
                                  _p(ne["W"], P_f64), _p(ne["gc"], P_f64), _p(ne["gp"], P_f64),
                                  _p(ext["obs_mask"], P_u8), _p(ext["cam_rank"], P_i32),
                                  _p(ext["pt_rank"], P_i32), ext["n_cam_free"], lam, _p(S, P_f64),
                                  _p(b, P_f64))
        return S, b

    def solve_step(self, ne, ext, lam):
        dc = np.zeros((self.n_cams, 9)); dp = np.zeros((self.n_pts, 3))
        pred, rr = ct.c_double(0), ct.c_double(0)
        st = self.L.oracle_solve_step(ct.byref(self._pb), self._o(), _p(ne["U"], P_f64),
                                      _p(ne["V"], P_f64), _p(ne["W"], P_f64), _p(ne["gc"], P_f64),
                                      _p(ne["gp"], P_f64), _p(ext["obs_mask"], P_u8),
                                      _p(ext["cam_rank"], P_i32), _p(ext["pt_rank"], P_i32),
                                      ext["n_cam_free"], lam, _p(dc, P_f64), _p(dp, P_f64),
                                      ct.byref(pred), ct.byref(rr))
        return dict(status=st, dc=dc, dp=dp, pred_decrease=pred.value, pcg_rel_res=rr.value)

    def apply_step(self, cams, pts, dc, dp):
        cams, pts = _f64(cams), _f64(pts)
        co = np.zeros_like(cams); po = np.zeros_like(pts)
        self.L.oracle_apply_step(self.n_cams, self.n_pts, _p(cams, P_f64), _p(pts, P_f64),
                                 _p(_f64(dc), P_f64), _p(_f64(dp), P_f64), _p(co, P_f64), _p(po, P_f64))
        return co, po

    def lm(self, cams0, pts0, max_iters, alive=None):
        cams = _f64(cams0).copy()
        pts = _f64(pts0).copy()
        log = (IterLog * max(1, max_iters))()
        al = None if alive is None else np.ascontiguousarray(alive, dtype=np.uint8)
        n = self.L.oracle_lm(ct.byref(self._pb), self._o(), int(max_iters), _p(cams, P_f64),
                             _p(pts, P_f64), log, None if al is None else _p(al, P_u8))
        rows = []
        for i in range(n):
            e = log[i]
            rows.append(dict(cost=e.cost, rmse_px=e.rmse_px, lam=e.lambda_, gain=e.gain,
                             pred_decrease=e.pred_decrease, cand_cost=e.cand_cost,
                             accepted=bool(e.accepted), pcg_iters=e.pcg_iters,
                             pcg_rel_res=e.pcg_rel_res, n_cam_act=e.n_cam_act,
                             n_pt_act=e.n_pt_act, n_obs_act=e.n_obs_act))
        return cams, pts, rows

    def backward(self, cams, pts, ext, dL_dcams, dL_dpts):
        duv = np.zeros((self.n_obs, 2)); dd = np.zeros(self.n_obs)
        st = self.L.oracle_backward(ct.byref(self._pb), self._o(), _p(_f64(cams), P_f64),
                                    _p(_f64(pts), P_f64), _p(ext["obs_mask"], P_u8),
                                    _p(ext["cam_rank"], P_i32), _p(ext["pt_rank"], P_i32),
                                    ext["n_cam_free"], _p(_f64(dL_dcams), P_f64),
                                    _p(_f64(dL_dpts), P_f64), _p(duv, P_f64), _p(dd, P_f64))
        if st != 0:
            raise RuntimeError("oracle backward: factorisation failed")
        return duv, dd


@dataclasses.dataclass
class OracleGPOptions:
    huber_delta: float = 0.1
    lambda0: float = 1e-4

    def to_c(self) -> GPOpts:
        return GPOpts(**dataclasses.asdict(self))


class OracleGP:
    """Depth-constrained global positioning (Sec. 3.1, 4.1) of one problem, host arrays
    in input order; scales are full-length [N] (pinned entries are ignored)."""

    def __init__(self, n_cams, n_pts, obs_cam, obs_pt, rays, depth, fixed_cams=(0,),
                 opts: OracleGPOptions | None = None):
        self.L = lib()
        self.n_cams, self.n_pts = int(n_cams), int(n_pts)
        self.obs_cam = np.ascontiguousarray(obs_cam, dtype=np.int32)
        self.obs_pt = np.ascontiguousarray(obs_pt, dtype=np.int32)
        self.rays = _f64(rays).reshape(-1, 3)
        self.depth = _f64(depth)
        self.fixed = np.zeros(self.n_cams, dtype=np.uint8)
        self.fixed[np.asarray(fixed_cams, dtype=np.int64)] = 1
        self.n_obs = int(self.obs_cam.shape[0])
        self.opts = opts or OracleGPOptions()
        self._pb = GPProblem(self.n_cams, self.n_pts, self.n_obs, _p(self.obs_cam, P_i32),
                             _p(self.obs_pt, P_i32), _p(self.rays, P_f64), _p(self.depth, P_f64),
                             _p(self.fixed, P_u8))

    @classmethod
    def from_scene(cls, sc, opts: OracleGPOptions | None = None):
        return cls(sc.centres0.shape[0], sc.pts0.shape[0], sc.obs_cam, sc.obs_pt, sc.rays, sc.depth,
                   sc.fixed_cams, opts)

    def _o(self):
        return ct.byref(self.opts.to_c())

    def free_set(self):
        fr = np.zeros(self.n_obs, np.int32)
        n = self.L.oracle_gp_free_set(ct.byref(self._pb), _p(fr, P_i32))
        return fr, int(n)

    def cost(self, centres, pts, scales):
        rms = ct.c_double(0)
        F = self.L.oracle_gp_cost(ct.byref(self._pb), self._o(), _p(_f64(centres), P_f64),
                                  _p(_f64(pts), P_f64), _p(_f64(scales), P_f64), ct.byref(rms))
        return F, rms.value

    def normal_equations(self, centres, pts, scales):
        C, P, N = self.n_cams, self.n_pts, self.n_obs
        out = dict(U=np.zeros((C, 3, 3)), V=np.zeros((P, 3, 3)), W=np.zeros((N, 3, 3)),
                   Hts=np.zeros((N, 3)), HXs=np.zeros((N, 3)), Q=np.zeros(N), gt=np.zeros((C, 3)),
                   gX=np.zeros((P, 3)), gs=np.zeros(N))
        self.L.oracle_gp_normal_equations(ct.byref(self._pb), self._o(), _p(_f64(centres), P_f64),
                                          _p(_f64(pts), P_f64), _p(_f64(scales), P_f64),
                                          *[_p(out[k], P_f64) for k in ("U", "V", "W", "Hts", "HXs", "Q",
                                                                        "gt", "gX", "gs")])
        return out

    def solve_step(self, centres, pts, scales, lam):
        dt = np.zeros((self.n_cams, 3)); dX = np.zeros((self.n_pts, 3)); ds = np.zeros(self.n_obs)
        pred = ct.c_double(0)
        st = self.L.oracle_gp_solve_step(ct.byref(self._pb), self._o(), _p(_f64(centres), P_f64),
                                         _p(_f64(pts), P_f64), _p(_f64(scales), P_f64), float(lam),
                                         _p(dt, P_f64), _p(dX, P_f64), _p(ds, P_f64), ct.byref(pred))
        return dict(status=st, dt=dt, dX=dX, ds=ds, pred_decrease=pred.value)

    def lm(self, centres0, pts0, scales0, max_iters):
        t = _f64(centres0).copy(); X = _f64(pts0).copy(); s = _f64(scales0).copy()
        log = (IterLog * max(1, max_iters))()
        n = self.L.oracle_gp_lm(ct.byref(self._pb), self._o(), int(max_iters), _p(t, P_f64),
                                _p(X, P_f64), _p(s, P_f64), log)
        rows = [dict(cost=log[i].cost, rms=log[i].rmse_px, lam=log[i].lambda_, gain=log[i].gain,
                     pred_decrease=log[i].pred_decrease, cand_cost=log[i].cand_cost,
                     accepted=bool(log[i].accepted), n_cam_free=log[i].n_cam_act,
                     n_pt_act=log[i].n_pt_act, n_free=log[i].n_obs_act) for i in range(n)]
        return t, X, s, rows


def gp_residual(t, X, v, s):
    u = np.zeros(3); Jt = np.zeros(9); JX = np.zeros(9); Js = np.zeros(3)
    lib().oracle_gp_residual(_p(_f64(t), P_f64), _p(_f64(X), P_f64), _p(_f64(v), P_f64), float(s),
                             _p(u, P_f64), _p(Jt, P_f64), _p(JX, P_f64), _p(Js, P_f64))
    return u, Jt.reshape(3, 3), JX.reshape(3, 3), Js


def rotvec_to_matrix(w):
    R = np.zeros(9)
    lib().oracle_rotvec_to_matrix(_p(_f64(w), P_f64), _p(R, P_f64))
    return R.reshape(3, 3)


def so3_left_jacobian_inv(w):
    J = np.zeros(9)
    lib().oracle_so3_left_jacobian_inv(_p(_f64(w), P_f64), _p(J, P_f64))
    return J.reshape(3, 3)


def rotvec_compose(a, b):
    o = np.zeros(3)
    lib().oracle_rotvec_compose(_p(_f64(a), P_f64), _p(_f64(b), P_f64), _p(o, P_f64))
    return o


def observe(cam, X, uv, tau, wt, cx=320.0, cy=240.0, model=0):
    r = np.zeros(3); Jc = np.zeros(27); Jp = np.zeros(9); z = ct.c_double(0); uvh = np.zeros(2)
    lib().oracle_observe_model(int(model), _p(_f64(cam), P_f64), _p(_f64(X), P_f64), _p(_f64(uv), P_f64),
                               tau, wt, cx, cy, _p(r, P_f64), _p(Jc, P_f64), _p(Jp, P_f64), ct.byref(z),
                               _p(uvh, P_f64))
    return r, Jc.reshape(3, 9), Jp.reshape(3, 3), z.value, uvh


def lm_accept(F, Fc, pred) -> bool:
    return bool(lib().oracle_lm_accept(float(F), float(Fc), float(pred)))


def lm_damping(accepted, gain, lam, nu):
    """One damping update; returns (lambda, nu) after the step."""
    a, b = ct.c_double(lam), ct.c_double(nu)
    lib().oracle_lm_damping(int(bool(accepted)), float(gain), ct.byref(a), ct.byref(b))
    return a.value, b.value


def set_threads(n: int):
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())
