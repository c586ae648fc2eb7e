"""Python binding of the C ABI in include/ba_b300.h (libba_b300.so).

Argument marshalling only: every step of the LM iteration runs in the
library's CUDA kernels.  Arrays may be NumPy arrays (host memory) or torch
tensors (host or CUDA); the library copies through unified addressing.
Importing this module never falls back to a CPU implementation: if the
shared library is missing or cannot be loaded, it raises.
"""
from __future__ import annotations

import ctypes as ct
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BA_DEBUG_BOUNDS=1 selects the build with the device index checks (ba_debug_bounds)
LIB_PATH = os.path.join(_HERE, "libba_b300_debug.so" if os.environ.get("BA_DEBUG_BOUNDS") == "1"
                        else "libba_b300.so")

BA_OK, BA_ERR_INVALID_ARG, BA_ERR_CUDA, BA_ERR_OOM = 0, 1, 2, 3
BA_ERR_NOT_CONVERGED, BA_ERR_NONFINITE, BA_ERR_STATE, BA_ERR_TIMEOUT = 4, 5, 6, 7
BA_FP64, BA_FP32 = 0, 1
BA_SOLVER_AUTO, BA_SOLVER_IMPLICIT, BA_SOLVER_EXPLICIT, BA_SOLVER_DENSE, BA_SOLVER_SPARSE = 0, 1, 2, 3, 4
BA_EXTRACT_DYNAMIC, BA_EXTRACT_ONCE = 0, 1
BA_CAMERA_RADIAL, BA_CAMERA_CENTRE = 0, 1

# every symbol include/ba_b300.h declares
EXPORTS = ("ba_default_options", "ba_create", "ba_lm_step", "ba_solve", "ba_get_params",
           "ba_set_params", "ba_get_active", "ba_extract", "ba_linearize", "ba_solve_damped",
           "ba_eval_cost", "ba_backward", "ba_eval_cost_noalloc", "ba_tc_gemm_nt", "ba_dense_cholesky",
           "ba_get_state", "ba_set_state", "ba_selftest_wait_timeout", "ba_selftest_layout",
           "ba_kernel_launches", "ba_debug_bounds", "ba_solver_kind", "ba_explicit_layout", "ba_formation_kernel", "ba_destroy", "ba_release_cache",
           "ba_status_string", "ba_last_error",
           "ba_gp_default_options", "ba_gp_create", "ba_gp_lm_step", "ba_gp_solve", "ba_gp_get_params",
           "ba_gp_get_free", "ba_gp_solve_damped", "ba_gp_eval_cost", "ba_gp_kernel_launches",
           "ba_gp_destroy")


class _Options(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("img_w", ct.c_int), ("img_h", ct.c_int),
                ("cx", ct.c_double), ("cy", ct.c_double), ("huber_delta", ct.c_double),
                ("depth_weight", ct.c_double), ("invalid_depth_weight", ct.c_double),
                ("min_depth", ct.c_double), ("extract_every", ct.c_int),
                ("drop_residual_px", ct.c_double), ("min_cam_obs", ct.c_int),
                ("min_pt_obs", ct.c_int), ("lambda0", ct.c_double), ("pcg_rel_tol", ct.c_double),
                ("pcg_max_iters", ct.c_int), ("fixed_cams", ct.POINTER(ct.c_int32)),
                ("n_fixed", ct.c_int), ("solver", ct.c_int), ("extract_mode", ct.c_int),
                ("camera_model", ct.c_int)]


class _GPOptions(ct.Structure):
    _fields_ = [("huber_delta", ct.c_double), ("lambda0", ct.c_double), ("pcg_rel_tol", ct.c_double),
                ("pcg_max_iters", ct.c_int), ("fixed_cams", ct.POINTER(ct.c_int32)), ("n_fixed", ct.c_int),
                ("solver", ct.c_int)]


class _IterInfo(ct.Structure):
    _fields_ = [("cost", ct.c_double), ("rmse_px", ct.c_double), ("lambda_", ct.c_double),
                ("gain", ct.c_double), ("pred_decrease", ct.c_double), ("cand_cost", ct.c_double),
                ("accepted", ct.c_int), ("pcg_iters", ct.c_int), ("pcg_rel_res", ct.c_double),
                ("n_cam_act", ct.c_int64), ("n_pt_act", ct.c_int64), ("n_obs_act", ct.c_int64),
                ("ms", ct.c_float * 8)]

    def as_dict(self):
        return dict(cost=self.cost, rmse_px=self.rmse_px, lam=self.lambda_, gain=self.gain,
                    pred_decrease=self.pred_decrease, cand_cost=self.cand_cost,
                    accepted=bool(self.accepted), pcg_iters=self.pcg_iters,
                    pcg_rel_res=self.pcg_rel_res, n_cam_act=self.n_cam_act,
                    n_pt_act=self.n_pt_act, n_obs_act=self.n_obs_act, ms=list(self.ms))


_lib = None


def lib():
    """Load libba_b300.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2510_13310_b300.build` (no CPU fallback exists)")
        try:  # torch first, so the CUDA runtime it loads is the one shared with the library
            import torch  # noqa: F401
        except ImportError:
            pass
        L = ct.CDLL(LIB_PATH)
        vp = ct.c_void_p
        L.ba_default_options.argtypes = [ct.POINTER(_Options)]
        L.ba_create.argtypes = [ct.POINTER(_Options), vp, ct.c_int64, vp, ct.c_int64, vp, ct.c_int64,
                                vp, vp, vp, vp, ct.POINTER(vp)]
        L.ba_lm_step.argtypes = [vp, ct.POINTER(_IterInfo)]
        L.ba_solve.argtypes = [vp, ct.c_int, ct.POINTER(_IterInfo), ct.POINTER(ct.c_int)]
        L.ba_get_params.argtypes = [vp, vp, vp]
        L.ba_set_params.argtypes = [vp, vp, vp]
        L.ba_get_active.argtypes = [vp, vp, vp, vp, vp, vp]
        L.ba_extract.argtypes = [vp, ct.c_int, ct.POINTER(ct.c_int)]
        L.ba_linearize.argtypes = [vp, vp, vp, vp, vp, vp]
        L.ba_solve_damped.argtypes = [vp, ct.c_double, vp, vp, ct.POINTER(_IterInfo)]
        L.ba_eval_cost.argtypes = [vp, vp, vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
        L.ba_backward.argtypes = [vp, vp, vp, vp, vp]
        L.ba_debug_bounds.argtypes = [ct.c_int, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64)]
        L.ba_eval_cost_noalloc.argtypes = [ct.POINTER(_Options), vp, ct.c_int64, vp, ct.c_int64, vp,
                                           ct.c_int64, vp, vp, vp, vp, vp, vp]
        L.ba_kernel_launches.argtypes = [vp]
        L.ba_kernel_launches.restype = ct.c_int64
        L.ba_solver_kind.argtypes = [vp]
        L.ba_solver_kind.restype = ct.c_int
        L.ba_explicit_layout.argtypes = [vp, vp, vp, vp]
        L.ba_explicit_layout.restype = None
        L.ba_formation_kernel.argtypes = [vp]
        L.ba_formation_kernel.restype = ct.c_int
        L.ba_get_state.argtypes = [vp, vp, ct.POINTER(ct.c_size_t)]
        L.ba_set_state.argtypes = [vp, vp, ct.c_size_t]
        L.ba_selftest_wait_timeout.argtypes = [vp, ct.c_double]
        L.ba_selftest_layout.argtypes = [ct.c_int64, vp, ct.c_int64, vp, ct.c_int64, vp, vp, vp, ct.c_int,
                                         ct.POINTER(ct.c_int)]
        L.ba_tc_gemm_nt.argtypes = [vp, ct.c_int64, ct.c_int64, ct.c_int64, ct.c_float, vp, ct.c_int64, vp,
                                    ct.c_int64, ct.c_float, vp, ct.c_int64]
        L.ba_dense_cholesky.argtypes = [vp, ct.c_int64, vp, ct.c_int64, vp, ct.c_int64, ct.POINTER(ct.c_int)]
        L.ba_destroy.argtypes = [vp]
        L.ba_release_cache.argtypes = []
        L.ba_release_cache.restype = None
        L.ba_gp_default_options.argtypes = [ct.POINTER(_GPOptions)]
        L.ba_gp_default_options.restype = None
        L.ba_gp_create.argtypes = [ct.POINTER(_GPOptions), vp, ct.c_int64, vp, ct.c_int64, vp, ct.c_int64,
                                   vp, vp, vp, vp, vp, ct.POINTER(ct.c_void_p)]
        L.ba_gp_lm_step.argtypes = [vp, ct.POINTER(_IterInfo)]
        L.ba_gp_solve.argtypes = [vp, ct.c_int, ct.POINTER(_IterInfo), ct.POINTER(ct.c_int)]
        L.ba_gp_get_params.argtypes = [vp, vp, vp, vp]
        L.ba_gp_get_free.argtypes = [vp, vp, ct.POINTER(ct.c_int64)]
        L.ba_gp_solve_damped.argtypes = [vp, ct.c_double, vp, vp, vp, ct.POINTER(_IterInfo)]
        L.ba_gp_eval_cost.argtypes = [vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
        L.ba_gp_kernel_launches.argtypes = [vp]
        L.ba_gp_kernel_launches.restype = ct.c_int64
        L.ba_gp_destroy.argtypes = [vp]
        L.ba_gp_destroy.restype = None
        L.ba_status_string.argtypes = [ct.c_int]
        L.ba_status_string.restype = ct.c_char_p
        L.ba_last_error.restype = ct.c_char_p
        for f in ("ba_create", "ba_lm_step", "ba_solve", "ba_get_params", "ba_set_params",
                  "ba_get_active", "ba_extract", "ba_linearize", "ba_solve_damped", "ba_eval_cost",
                  "ba_backward", "ba_eval_cost_noalloc", "ba_tc_gemm_nt", "ba_dense_cholesky",
                  "ba_get_state", "ba_set_state", "ba_selftest_wait_timeout", "ba_selftest_layout",
                  "ba_gp_create", "ba_gp_lm_step", "ba_gp_solve", "ba_gp_get_params", "ba_gp_get_free",
                  "ba_gp_solve_damped", "ba_gp_eval_cost"):
            getattr(L, f).restype = ct.c_int
        _lib = L
    return _lib


class BAError(RuntimeError):
    def __init__(self, status, where):
        L = lib()
        msg = L.ba_status_string(status).decode()
        detail = L.ba_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")
        self.status = status


def _check(status, where, allow=(BA_OK,)):
    if status not in allow:
        raise BAError(status, where)
    return status


@dataclasses.dataclass
class Options:
    precision: int = BA_FP32
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
    fixed_cams: tuple = (0,)
    solver: int = BA_SOLVER_AUTO
    extract_mode: int = 0  # BA_EXTRACT_DYNAMIC; 1 = BA_EXTRACT_ONCE (one-shot pruning)
    camera_model: int = 0  # BA_CAMERA_RADIAL; 1 = BA_CAMERA_CENTRE (centre + rotation + focal)


class _Arr:
    """Keeps a host/device buffer alive and exposes its address.

    size: the element count the library will read or write (ValueError otherwise:
    the C ABI takes bare pointers and cannot check).  out: the library writes into
    the buffer, so it must be used in place: the exact dtype, contiguous (a NumPy
    array also writeable); anything that would need a converted copy is refused
    instead of silently receiving the results in a temporary."""

    def __init__(self, a, dtype, size=None, what="array", out=False):
        self.obj = a
        if hasattr(a, "data_ptr"):  # torch tensor
            import torch
            tdt = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8,
                   np.float32: torch.float32}[dtype]
            if out and (a.dtype != tdt or not a.is_contiguous()):
                raise ValueError(f"{what}: output tensor must be contiguous {tdt}")
            t = a.contiguous()
            if t.dtype != tdt:
                t = t.to(tdt)
            self.obj = t
            self.ptr = t.data_ptr()
            n = t.numel()
        else:
            if out and not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous
                            and a.flags.writeable):
                raise ValueError(f"{what}: output array must be a writeable C-contiguous {np.dtype(dtype)} array")
            arr = np.ascontiguousarray(a, dtype=dtype)
            self.obj = arr
            self.ptr = arr.ctypes.data
            n = arr.size
        if size is not None and n != size:
            raise ValueError(f"{what}: {n} elements, expected {size}")
        self.n = n

    @property
    def p(self):
        return ct.c_void_p(self.ptr)


def release_cache():
    """ba_release_cache: return the device buffers of destroyed problems to the driver."""
    lib().ba_release_cache()


def selftest_layout(cams, pts, obs_cam, obs_pt, obs_uv, with_covis=True):
    """ba_selftest_layout on host arrays: the mismatch bitmask (0 = the device
    layout equals the host reference layout bit for bit)."""
    L = lib()
    arrs = _problem_arrays(cams, pts, obs_cam, obs_pt, obs_uv, None)
    mm = ct.c_int(-1)
    _check(L.ba_selftest_layout(arrs[0].n // 9, arrs[0].p, arrs[1].n // 3, arrs[1].p, arrs[2].n,
                                arrs[2].p, arrs[3].p, arrs[4].p, int(bool(with_covis)), ct.byref(mm)),
           "ba_selftest_layout")
    return mm.value


def _problem_arrays(cams, pts, obs_cam, obs_pt, obs_uv, depth, cam_width=9, uv_width=2, what="ba_create"):
    """The input arrays of a problem, sizes checked against each other: cams
    [C][cam_width], pts [P][3], obs_cam, obs_pt [N], obs_uv [N][uv_width], depth [N]."""
    c = _Arr(cams, np.float64, what=f"{what}: cameras")
    p = _Arr(pts, np.float64, what=f"{what}: points")
    if c.n % cam_width or p.n % 3:
        raise ValueError(f"{what}: camera array of {c.n} values is not [C][{cam_width}] "
                         f"or point array of {p.n} values is not [P][3]")
    oc = _Arr(obs_cam, np.int32, what=f"{what}: obs_cam")
    N = oc.n
    arrs = [c, p, oc, _Arr(obs_pt, np.int32, N, f"{what}: obs_pt"),
            _Arr(obs_uv, np.float64, uv_width * N, f"{what}: observations")]
    if depth is not None:
        arrs.append(_Arr(depth, np.float64, N, f"{what}: depth"))
    return arrs


def _stream_handle(stream):
    if stream is not None:
        return ct.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ct.c_void_p(0)


class Problem:
    """One bundle-adjustment problem living on the current CUDA device."""

    def __init__(self, cams, pts, obs_cam, obs_pt, obs_uv, depth, options: Options | None = None,
                 stream=None):
        self.L = lib()
        self.options = options or Options()
        o = self.options
        copt, self._fixed = _c_options(o)
        arrs = _problem_arrays(cams, pts, obs_cam, obs_pt, obs_uv, depth)
        self.n_cams = arrs[0].n // 9
        self.n_pts = arrs[1].n // 3
        self.n_obs = arrs[2].n
        h = ct.c_void_p()
        st = self.L.ba_create(ct.byref(copt), _stream_handle(stream), self.n_cams, arrs[0].p,
                              self.n_pts, arrs[1].p, self.n_obs, arrs[2].p, arrs[3].p, arrs[4].p,
                              arrs[5].p, ct.byref(h))
        _check(st, "ba_create")
        self.h = h

    @classmethod
    def from_scene(cls, scene, options: Options | None = None, stream=None):
        opts = options or Options()
        if tuple(opts.fixed_cams) != tuple(int(c) for c in scene.fixed_cams):
            opts = dataclasses.replace(opts, fixed_cams=tuple(int(c) for c in scene.fixed_cams))
        return cls(scene.cams0, scene.pts0, scene.obs_cam, scene.obs_pt, scene.obs_uv, scene.depth,
                   opts, stream)

    def close(self):
        if getattr(self, "h", None):
            self.L.ba_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lm_step(self):
        info = _IterInfo()
        _check(self.L.ba_lm_step(self.h, ct.byref(info)), "ba_lm_step",
               allow=(BA_OK, BA_ERR_NOT_CONVERGED, BA_ERR_NONFINITE))
        return info.as_dict()

    def solve(self, max_iters):
        log = (_IterInfo * max(1, max_iters))()
        n = ct.c_int(0)
        _check(self.L.ba_solve(self.h, int(max_iters), log, ct.byref(n)), "ba_solve",
               allow=(BA_OK, BA_ERR_NOT_CONVERGED))
        return [log[i].as_dict() for i in range(n.value)]

    def get_params(self, cams=None, pts=None):
        """Copies into the given buffers (NumPy or torch); allocates NumPy arrays if omitted."""
        c = cams if cams is not None else np.zeros((self.n_cams, 9))
        p = pts if pts is not None else np.zeros((self.n_pts, 3))
        ca = _Arr(c, np.float64, 9 * self.n_cams, "get_params: cameras", out=True)
        pa = _Arr(p, np.float64, 3 * self.n_pts, "get_params: points", out=True)
        _check(self.L.ba_get_params(self.h, ca.p, pa.p), "ba_get_params")
        return ca.obj, pa.obj

    def set_params(self, cams, pts):
        ca = _Arr(cams, np.float64, 9 * self.n_cams, "set_params: cameras")
        pa = _Arr(pts, np.float64, 3 * self.n_pts, "set_params: points")
        _check(self.L.ba_set_params(self.h, ca.p, pa.p), "ba_set_params")

    def extract(self, drop=False):
        n = ct.c_int(0)
        _check(self.L.ba_extract(self.h, 1 if drop else 0, ct.byref(n)), "ba_extract")
        return n.value

    def get_active(self):
        cm = np.zeros(self.n_cams, np.uint8)
        pm = np.zeros(self.n_pts, np.uint8)
        om = np.zeros(self.n_obs, np.uint8)
        cr = np.zeros(self.n_cams, np.int32)
        pr = np.zeros(self.n_pts, np.int32)
        _check(self.L.ba_get_active(self.h, cm.ctypes.data, pm.ctypes.data, om.ctypes.data,
                                    cr.ctypes.data, pr.ctypes.data), "ba_get_active")
        return dict(cam_mask=cm, pt_mask=pm, obs_mask=om, cam_rank=cr, pt_rank=pr)

    def linearize(self, want_W=True):
        U = np.zeros((self.n_cams, 9, 9)); V = np.zeros((self.n_pts, 3, 3))
        gc = np.zeros((self.n_cams, 9)); gp = np.zeros((self.n_pts, 3))
        W = np.zeros((self.n_obs, 9, 3)) if want_W else None
        _check(self.L.ba_linearize(self.h, U.ctypes.data, V.ctypes.data,
                                   W.ctypes.data if want_W else None, gc.ctypes.data, gp.ctypes.data),
               "ba_linearize")
        return dict(U=U, V=V, W=W, gc=gc, gp=gp)

    def solve_damped(self, lam):
        dc = np.zeros((self.n_cams, 9)); dp = np.zeros((self.n_pts, 3))
        info = _IterInfo()
        _check(self.L.ba_solve_damped(self.h, float(lam), dc.ctypes.data, dp.ctypes.data,
                                      ct.byref(info)), "ba_solve_damped")
        d = info.as_dict()
        d.update(dc=dc, dp=dp)
        return d

    def eval_cost(self, cams=None, pts=None):
        F, r = ct.c_double(0), ct.c_double(0)
        ca = _Arr(cams, np.float64, 9 * self.n_cams, "eval_cost: cameras") if cams is not None else None
        pa = _Arr(pts, np.float64, 3 * self.n_pts, "eval_cost: points") if pts is not None else None
        _check(self.L.ba_eval_cost(self.h, ca.p if ca else None, pa.p if pa else None,
                                   ct.byref(F), ct.byref(r)), "ba_eval_cost")
        return F.value, r.value

    def backward(self, dL_dcams, dL_dpts, dL_duv=None, dL_ddepth=None):
        duv = dL_duv if dL_duv is not None else np.zeros((self.n_obs, 2))
        dd = dL_ddepth if dL_ddepth is not None else np.zeros(self.n_obs)
        a = _Arr(dL_dcams, np.float64, 9 * self.n_cams, "backward: dL/dcams")
        b = _Arr(dL_dpts, np.float64, 3 * self.n_pts, "backward: dL/dpts")
        ua = _Arr(duv, np.float64, 2 * self.n_obs, "backward: dL/duv", out=True)
        da = _Arr(dd, np.float64, self.n_obs, "backward: dL/ddepth", out=True)
        _check(self.L.ba_backward(self.h, a.p, b.p, ua.p, da.p), "ba_backward",
               allow=(BA_OK, BA_ERR_NOT_CONVERGED))
        return ua.obj, da.obj

    def get_state(self) -> bytes:
        """ba_get_state: a checkpoint of the LM run (parameters, damping, iteration, drop bits)."""
        n = ct.c_size_t(0)
        _check(self.L.ba_get_state(self.h, None, ct.byref(n)), "ba_get_state")
        buf = (ct.c_ubyte * n.value)()
        _check(self.L.ba_get_state(self.h, ct.cast(buf, ct.c_void_p), ct.byref(n)), "ba_get_state")
        return bytes(buf)

    def set_state(self, blob: bytes):
        """ba_set_state: resume from a checkpoint taken on a problem with the same observations."""
        buf = (ct.c_ubyte * len(blob)).from_buffer_copy(blob)
        _check(self.L.ba_set_state(self.h, ct.cast(buf, ct.c_void_p), len(blob)), "ba_set_state")

    @property
    def kernel_launches(self):
        return int(self.L.ba_kernel_launches(self.h))

    @property
    def solver_kind(self) -> int:
        """BA_SOLVER_IMPLICIT, BA_SOLVER_EXPLICIT or BA_SOLVER_DENSE (ba_solver_kind)."""
        return int(self.L.ba_solver_kind(self.h))

    @property
    def formation_kernel(self) -> str | None:
        """ba_formation_kernel: the kernel forming the explicit system's blocks."""
        return {1: "k_form_S_runs", 2: "k_form_S_lanes", 3: "k_form_S_cam", 4: "k_form_S_rec"}.get(self.L.ba_formation_kernel(self.h))

    @property
    def explicit_layout(self) -> dict:
        """ba_explicit_layout: where the explicit solver keeps S^ rows and PCG vectors."""
        r, v, g = ct.c_int(0), ct.c_int(0), ct.c_int(0)
        self.L.ba_explicit_layout(self.h, ct.byref(r), ct.byref(v), ct.byref(g))
        return {"rows_in_smem": r.value, "vecs_in_smem": v.value, "grid": g.value}

    @property
    def explicit_solver(self) -> bool:
        """True when the reduced camera system is formed explicitly (BA_SOLVER_EXPLICIT)."""
        return int(self.L.ba_solver_kind(self.h)) == BA_SOLVER_EXPLICIT


def _c_options(o: Options):
    fixed = np.ascontiguousarray(np.asarray(o.fixed_cams, dtype=np.int32))
    c = _Options(o.precision, o.img_w, o.img_h, o.cx, o.cy, o.huber_delta, o.depth_weight,
                 o.invalid_depth_weight, o.min_depth, o.extract_every, o.drop_residual_px,
                 o.min_cam_obs, o.min_pt_obs, o.lambda0, o.pcg_rel_tol, o.pcg_max_iters,
                 fixed.ctypes.data_as(ct.POINTER(ct.c_int32)), len(fixed), o.solver, o.extract_mode,
                 o.camera_model)
    return c, fixed


def paper_cameras(centres, quats, focal):
    """Cameras in the parameterisation of Sec. 3.2 (centre c [C,3], unit quaternion
    (w, x, y, z) of the world-to-camera rotation [C,4], focal [C]) as the library's
    nine slots under BA_CAMERA_CENTRE: [axis-angle of the rotation, c, f, 0, 0]."""
    from scipy.spatial.transform import Rotation
    q = np.asarray(quats, dtype=np.float64)
    rv = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1)).as_rotvec()
    C = q.shape[0]
    return np.concatenate([rv, np.asarray(centres, np.float64).reshape(C, 3),
                           np.asarray(focal, np.float64).reshape(C, 1), np.zeros((C, 2))], axis=1)


def paper_cameras_from(cams):
    """The inverse of paper_cameras: (centres, quaternions (w, x, y, z), focal)."""
    from scipy.spatial.transform import Rotation
    cams = np.asarray(cams, dtype=np.float64)
    xyzw = Rotation.from_rotvec(cams[:, :3]).as_quat()
    return cams[:, 3:6].copy(), np.stack([xyzw[:, 3], xyzw[:, 0], xyzw[:, 1], xyzw[:, 2]], 1), cams[:, 6].copy()


def _check_noalloc_args(cams, pts, obs_cam, obs_pt, obs_uv, depth, out, obs_mask):
    """Types, layout and sizes of ba_eval_cost_noalloc's tensors (the C ABI takes
    bare pointers and cannot check them).  Raises ValueError."""
    import torch

    spec = [("cams", cams, torch.float64), ("pts", pts, torch.float64),
            ("obs_cam", obs_cam, torch.int32), ("obs_pt", obs_pt, torch.int32),
            ("obs_uv", obs_uv, torch.float64), ("depth", depth, torch.float64),
            ("out", out, torch.float64)]
    if obs_mask is not None:
        spec.append(("obs_mask", obs_mask, (torch.uint8, torch.bool)))
    for name, t, dt in spec:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"eval_cost_noalloc: {name} must be a torch tensor")
        ok = t.dtype in dt if isinstance(dt, tuple) else t.dtype == dt
        if not ok:
            raise ValueError(f"eval_cost_noalloc: {name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"eval_cost_noalloc: {name} must be contiguous")
    if cams.numel() % 9 or pts.numel() % 3:
        raise ValueError("eval_cost_noalloc: cams must hold [C][9] and pts [P][3] values")
    n = obs_cam.numel()
    if obs_pt.numel() != n or depth.numel() != n or obs_uv.numel() != 2 * n or (
            obs_mask is not None and obs_mask.numel() != n):
        raise ValueError("eval_cost_noalloc: obs_pt, depth, obs_mask need N entries and obs_uv 2N "
                         f"(N = {n})")
    if out.numel() < 3:
        raise ValueError("eval_cost_noalloc: out needs 3 entries")
    devs = {t.device for _, t, _ in spec}
    if len(devs) != 1 or next(iter(devs)).type != "cuda":
        raise ValueError("eval_cost_noalloc: every tensor must be on one CUDA device")
    if next(iter(devs)).index != torch.cuda.current_device():
        raise ValueError("eval_cost_noalloc: the tensors must be on the current CUDA device")


def eval_cost_noalloc(cams, pts, obs_cam, obs_pt, obs_uv, depth, out, obs_mask=None,
                      options: Options | None = None, stream=None):
    """ba_eval_cost_noalloc: every argument a contiguous CUDA tensor of the current
    device (cams/pts/obs_uv/depth/out float64, indices int32, obs_mask uint8 or bool,
    out with 3 entries); wrong types, layouts or sizes raise ValueError.  Enqueued
    on the stream; nothing is allocated."""
    _check_noalloc_args(cams, pts, obs_cam, obs_pt, obs_uv, depth, out, obs_mask)
    L = lib()
    copt, _fixed = _c_options(options or Options())
    n_cams = cams.numel() // 9
    n_pts = pts.numel() // 3
    n_obs = obs_cam.numel()
    st = L.ba_eval_cost_noalloc(ct.byref(copt), _stream_handle(stream), n_cams, cams.data_ptr(),
                                n_pts, pts.data_ptr(), n_obs, obs_cam.data_ptr(), obs_pt.data_ptr(),
                                obs_uv.data_ptr(), depth.data_ptr(),
                                None if obs_mask is None else obs_mask.data_ptr(), out.data_ptr())
    _check(st, "ba_eval_cost_noalloc")
    return out


@dataclasses.dataclass
class GPOptions:
    huber_delta: float = 0.1
    lambda0: float = 1e-4
    pcg_rel_tol: float = 1e-6
    pcg_max_iters: int = 500
    fixed_cams: tuple = (0,)
    solver: int = BA_SOLVER_AUTO  # or BA_SOLVER_EXPLICIT (block-Jacobi PCG), BA_SOLVER_DENSE (tensor cores)


class GPProblem:
    """Depth-constrained global positioning (ba_gp_*) on the current CUDA device:
    camera centres, points and the free per-observation scales."""

    def __init__(self, centres, pts, obs_cam, obs_pt, rays, depth, scales0=None,
                 options: GPOptions | None = None, stream=None):
        self.L = lib()
        o = self.options = options or GPOptions()
        self._fixed = np.ascontiguousarray(np.asarray(o.fixed_cams, dtype=np.int32))
        copt = _GPOptions(o.huber_delta, o.lambda0, o.pcg_rel_tol, o.pcg_max_iters,
                          self._fixed.ctypes.data_as(ct.POINTER(ct.c_int32)), len(self._fixed), o.solver)
        arrs = _problem_arrays(centres, pts, obs_cam, obs_pt, rays, depth, cam_width=3, uv_width=3,
                               what="ba_gp_create")
        self.n_cams = arrs[0].n // 3
        self.n_pts = arrs[1].n // 3
        self.n_obs = arrs[2].n
        s0 = None if scales0 is None else _Arr(scales0, np.float64, self.n_obs, "ba_gp_create: scales0")
        h = ct.c_void_p()
        _check(self.L.ba_gp_create(ct.byref(copt), _stream_handle(stream), self.n_cams, arrs[0].p, self.n_pts,
                                   arrs[1].p, self.n_obs, arrs[2].p, arrs[3].p, arrs[4].p, arrs[5].p,
                                   None if s0 is None else s0.p, ct.byref(h)), "ba_gp_create")
        self.h = h

    @classmethod
    def from_scene(cls, sc, options: GPOptions | None = None, stream=None):
        o = options or GPOptions()
        if tuple(o.fixed_cams) != tuple(int(c) for c in sc.fixed_cams):
            o = dataclasses.replace(o, fixed_cams=tuple(int(c) for c in sc.fixed_cams))
        return cls(sc.centres0, sc.pts0, sc.obs_cam, sc.obs_pt, sc.rays, sc.depth, sc.scales0, o, stream)

    def close(self):
        if getattr(self, "h", None):
            self.L.ba_gp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lm_step(self):
        info = _IterInfo()
        _check(self.L.ba_gp_lm_step(self.h, ct.byref(info)), "ba_gp_lm_step",
               allow=(BA_OK, BA_ERR_NOT_CONVERGED, BA_ERR_NONFINITE))
        return info.as_dict()

    def solve(self, max_iters):
        log = (_IterInfo * max(1, max_iters))()
        n = ct.c_int(0)
        _check(self.L.ba_gp_solve(self.h, int(max_iters), log, ct.byref(n)), "ba_gp_solve",
               allow=(BA_OK, BA_ERR_NOT_CONVERGED))
        return [log[i].as_dict() for i in range(n.value)]

    def get_params(self):
        c = np.zeros((self.n_cams, 3)); p = np.zeros((self.n_pts, 3)); s = np.zeros(self.n_obs)
        _check(self.L.ba_gp_get_params(self.h, c.ctypes.data, p.ctypes.data, s.ctypes.data), "ba_gp_get_params")
        return c, p, s

    def get_free(self):
        fr = np.zeros(self.n_obs, np.int32)
        n = ct.c_int64(0)
        _check(self.L.ba_gp_get_free(self.h, fr.ctypes.data, ct.byref(n)), "ba_gp_get_free")
        return fr, n.value

    def solve_damped(self, lam):
        dt = np.zeros((self.n_cams, 3)); dX = np.zeros((self.n_pts, 3)); ds = np.zeros(self.n_obs)
        info = _IterInfo()
        _check(self.L.ba_gp_solve_damped(self.h, float(lam), dt.ctypes.data, dX.ctypes.data, ds.ctypes.data,
                                         ct.byref(info)), "ba_gp_solve_damped")
        d = info.as_dict()
        return dict(dt=dt, dX=dX, ds=ds, pred_decrease=d["pred_decrease"], pcg_iters=d["pcg_iters"],
                    pcg_rel_res=d["pcg_rel_res"])

    def eval_cost(self):
        F, r = ct.c_double(0), ct.c_double(0)
        _check(self.L.ba_gp_eval_cost(self.h, ct.byref(F), ct.byref(r)), "ba_gp_eval_cost")
        return F.value, r.value

    @property
    def kernel_launches(self):
        return int(self.L.ba_gp_kernel_launches(self.h))


def _make_ba_function():
    import torch

    class BAFunction(torch.autograd.Function):
        """Differentiable bundle adjustment.

        forward(cams0 [C,9], pts0 [P,3], obs_uv [N,2], depth [N], obs_cam [N], obs_pt [N],
        options, iters) runs `iters` LM iterations (ba_solve) and returns the
        solution (cams [C,9], pts [P,3]) as float64 tensors on the inputs' device.
        backward gives dL/dobs_uv and dL/ddepth by the implicit adjoint at the
        solution (ba_backward); the gradients with respect to the initial
        parameters are zero, and the index arrays have none."""

        @staticmethod
        def forward(ctx, cams0, pts0, obs_uv, depth, obs_cam, obs_pt, options, iters):
            dev = obs_uv.device
            prob = Problem(cams0.detach(), pts0.detach(), obs_cam, obs_pt, obs_uv.detach(), depth.detach(),
                           options=options,
                           stream=torch.cuda.current_stream(dev).cuda_stream if dev.type == "cuda" else None)
            prob.solve(int(iters))
            cams = torch.empty((prob.n_cams, 9), dtype=torch.float64, device=dev)
            pts = torch.empty((prob.n_pts, 3), dtype=torch.float64, device=dev)
            prob.get_params(cams, pts)
            ctx.prob = prob
            ctx.uv_dtype, ctx.depth_dtype = obs_uv.dtype, depth.dtype
            return cams, pts

        @staticmethod
        def backward(ctx, g_cams, g_pts):
            prob = ctx.prob
            dev = g_cams.device
            duv = torch.empty((prob.n_obs, 2), dtype=torch.float64, device=dev)
            dd = torch.empty((prob.n_obs,), dtype=torch.float64, device=dev)
            prob.backward(g_cams.to(torch.float64).contiguous(), g_pts.to(torch.float64).contiguous(), duv, dd)
            prob.close()
            ctx.prob = None
            zc = torch.zeros_like(g_cams) if ctx.needs_input_grad[0] else None
            zp = torch.zeros_like(g_pts) if ctx.needs_input_grad[1] else None
            return (zc, zp, duv.to(ctx.uv_dtype), dd.to(ctx.depth_dtype), None, None, None, None)

    return BAFunction


_BAFunction = None


def bundle_adjust(cams0, pts0, obs_uv, depth, obs_cam, obs_pt, options: Options | None = None,
                  iters: int = 30):
    """LM bundle adjustment as a differentiable torch op (see BAFunction)."""
    global _BAFunction
    if _BAFunction is None:
        _BAFunction = _make_ba_function()
    return _BAFunction.apply(cams0, pts0, obs_uv, depth, obs_cam, obs_pt, options or Options(), iters)


def debug_bounds(reset=False):
    """The first failed device index check of a BA_DEBUG_BOUNDS build as (site,
    index); (0, 0) when none failed; (-1, 0) for the release library."""
    site, index = ct.c_int64(), ct.c_int64()
    _check(lib().ba_debug_bounds(1 if reset else 0, ct.byref(site), ct.byref(index)), "ba_debug_bounds")
    return site.value, index.value


def tc_gemm_nt(A, B, C=None, alpha=1.0, beta=0.0, stream=None):
    """ba_tc_gemm_nt: C = alpha A B^T + beta C on the tensor cores (TF32 inputs, FP32
    accumulation).  A [M,K], B [N,K], C [M,N]: contiguous float32 CUDA tensors."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float32, device=A.device)
    for t in (A, B, C):
        if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError("tc_gemm_nt: contiguous float32 CUDA tensors")
    L = lib()
    _check(L.ba_tc_gemm_nt(_stream_handle(stream), M, N, K, float(alpha), ct.c_void_p(A.data_ptr()), A.stride(0),
                           ct.c_void_p(B.data_ptr()), B.stride(0), float(beta), ct.c_void_p(C.data_ptr()),
                           C.stride(0)), "ba_tc_gemm_nt")
    return C


def dense_cholesky(A, stream=None):
    """ba_dense_cholesky: lower factor L of an SPD float32 matrix (NumPy or torch,
    host or device); returns L like A (NumPy in, NumPy out) and the flags."""
    n = A.shape[0]
    is_torch = hasattr(A, "data_ptr")
    if is_torch:
        import torch
        A = A.contiguous().to(torch.float32)
        Lo = torch.empty_like(A)
        pa, pl = A.data_ptr(), Lo.data_ptr()
    else:
        A = np.ascontiguousarray(A, dtype=np.float32)
        Lo = np.empty_like(A)
        pa, pl = A.ctypes.data, Lo.ctypes.data
    flags = ct.c_int(0)
    _check(lib().ba_dense_cholesky(_stream_handle(stream), n, ct.c_void_p(pa), n, ct.c_void_p(pl), n,
                                   ct.byref(flags)), "ba_dense_cholesky", allow=(BA_OK, BA_ERR_NONFINITE))
    return Lo, flags.value
