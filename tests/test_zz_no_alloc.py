"""ba_eval_cost_noalloc: the FP64 cost of a state for callers that cannot allocate
device memory (code under a framework that owns every device allocation, or with
a memory budget fixed at start-up).  It must agree with ba_eval_cost, the
problem-based entry point, and with the FP64 CPU oracle on the same state and
active set, call after call.

Kept in a file that pytest collects last, so a run that stops at the first
failure has already run every other test."""
import ctypes as ct

import numpy as np
import pytest

import oracle
from paper_2510_13310_b300 import ba, scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def test_noalloc_cost_matches_problem_cost_on_two_calls():
    sc = scenes.make_scene("small")
    opts = ba.Options(invalid_depth_weight=1e-3)
    prob = ba.Problem.from_scene(sc, opts)
    prob.extract()
    mask = prob.get_active()["obs_mask"]
    obs = [_dev(sc.obs_cam, torch.int32), _dev(sc.obs_pt, torch.int32),
           _dev(sc.obs_uv, torch.float64), _dev(sc.depth, torch.float64)]
    m = _dev(mask, torch.uint8)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    ob = oracle.OracleBA.from_scene(sc, oracle.OracleOptions(invalid_depth_weight=1e-3))
    for cams, pts in ((sc.cams0, sc.pts0), (sc.cams_gt, sc.pts_gt)):
        F_ref, rmse_ref = prob.eval_cost(cams, pts)
        F_or, rmse_or = ob.cost(cams, pts, mask)
        ba.eval_cost_noalloc(_dev(cams, torch.float64), _dev(pts, torch.float64), *obs, out,
                             obs_mask=m, options=opts)
        torch.cuda.synchronize()
        F, rmse, n = out.tolist()
        assert F == pytest.approx(F_ref, rel=1e-12)
        assert rmse == pytest.approx(rmse_ref, rel=1e-12)
        # FP64 on both sides, summed in different orders
        assert F == pytest.approx(F_or, rel=1e-12)
        assert rmse == pytest.approx(rmse_or, rel=1e-12)
        assert n == int(mask.sum())


def test_noalloc_rejects_oversize_and_unmapped_host_memory():
    L = ba.lib()
    copt, _fixed = ba._c_options(ba.Options())
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    C = 4097
    cams = torch.zeros((C, 9), dtype=torch.float64, device="cuda")
    pts = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    z_i = torch.zeros(1, dtype=torch.int32, device="cuda")
    z_d = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    st = L.ba_eval_cost_noalloc(ct.byref(copt), None, C, cams.data_ptr(), 1, pts.data_ptr(), 1,
                                z_i.data_ptr(), z_i.data_ptr(), z_d.data_ptr(), z_d.data_ptr(),
                                None, out.data_ptr())
    assert st == ba.BA_ERR_INVALID_ARG
    assert b"scratch limit" in L.ba_last_error()
    host = np.zeros((4, 9))
    st = L.ba_eval_cost_noalloc(ct.byref(copt), None, 4, host.ctypes.data, 1, pts.data_ptr(), 1,
                                z_i.data_ptr(), z_i.data_ptr(), z_d.data_ptr(), z_d.data_ptr(),
                                None, out.data_ptr())
    assert st == ba.BA_ERR_INVALID_ARG


def test_noalloc_call_captured_in_a_cuda_graph_replays_for_new_states():
    """The entry point exists for code captured into CUDA graphs: one call captured
    (after a warm-up call outside capture), then replayed with the cameras and
    points rewritten in place, must give ba_eval_cost's numbers each time."""
    sc = scenes.make_scene("small")
    opts = ba.Options(invalid_depth_weight=1e-3)
    prob = ba.Problem.from_scene(sc, opts)
    prob.extract()
    mask = prob.get_active()["obs_mask"]
    cams_d, pts_d = _dev(sc.cams0, torch.float64), _dev(sc.pts0, torch.float64)
    obs = [_dev(sc.obs_cam, torch.int32), _dev(sc.obs_pt, torch.int32),
           _dev(sc.obs_uv, torch.float64), _dev(sc.depth, torch.float64)]
    m = _dev(mask, torch.uint8)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ba.eval_cost_noalloc(cams_d, pts_d, *obs, out, obs_mask=m, options=opts, stream=side.cuda_stream)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ba.eval_cost_noalloc(cams_d, pts_d, *obs, out, obs_mask=m, options=opts,
                             stream=torch.cuda.current_stream().cuda_stream)
    for cams, pts in ((sc.cams_gt, sc.pts_gt), (sc.cams0, sc.pts0)):
        cams_d.copy_(torch.as_tensor(np.ascontiguousarray(cams)))
        pts_d.copy_(torch.as_tensor(np.ascontiguousarray(pts)))
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        F_ref, rmse_ref = prob.eval_cost(cams, pts)
        F, rmse, n = out.tolist()
        assert F == pytest.approx(F_ref, rel=1e-12)
        assert rmse == pytest.approx(rmse_ref, rel=1e-12)
        assert n == int(mask.sum())
