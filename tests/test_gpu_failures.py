"""Failure detection without faulting the GPU: a bounded device wait on a flag that
nothing sets gives up with a status the host reads and the context stays usable; a
PCG capped at one iteration reports BA_ERR_NOT_CONVERGED and still takes a step;
non-finite inputs are refused on the host."""
import ctypes as ct

import numpy as np
import pytest

from paper_2510_13310_b300 import ba, scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_bounded_wait_gives_up_and_context_survives():
    L = ba.lib()
    assert L.ba_selftest_wait_timeout(None, 10.0) == ba.BA_ERR_TIMEOUT
    assert "as intended" in L.ba_last_error().decode()
    # the context is intact: a tensor-core product and an LM step still run
    A = torch.randn(128, 64, device="cuda")
    C = ba.tc_gemm_nt(A, A)
    assert torch.allclose(C, A @ A.T, rtol=5e-3, atol=5e-2)
    sc = scenes.make_scene("small", scale=0.5)
    ba.Problem.from_scene(sc).lm_step()
    assert L.ba_selftest_wait_timeout(None, 0.0) == ba.BA_ERR_INVALID_ARG


@pytest.mark.parametrize("solver", [ba.BA_SOLVER_IMPLICIT, ba.BA_SOLVER_EXPLICIT])
def test_pcg_cap_reports_not_converged_and_still_steps(solver):
    sc = scenes.make_scene("small", scale=0.5)
    p = ba.Problem.from_scene(sc, ba.Options(pcg_max_iters=1, solver=solver))
    info = ba._IterInfo()
    st = p.L.ba_lm_step(p.h, ct.byref(info))
    d = info.as_dict()
    assert st == ba.BA_ERR_NOT_CONVERGED
    assert d["pcg_iters"] == 1 and d["pcg_rel_res"] > 1e-6
    assert np.isfinite(d["cand_cost"])


def test_nonfinite_parameters_refused():
    sc = scenes.make_scene("small", scale=0.5)
    p = ba.Problem.from_scene(sc)
    cams = sc.cams0.copy()
    cams[1, 4] = np.inf
    with pytest.raises(ba.BAError, match="invalid argument"):
        p.set_params(cams, sc.pts0)
    p.lm_step()  # the problem is unchanged and usable


@pytest.mark.parametrize("pinned", [False, True])
def test_create_from_host_arrays_reports_errors_in_check_order(pinned):
    """Host arrays: the indices upload first and are sorted while the values
    upload on a second stream and are checked there; a non-finite value is still
    reported before an index error, as when every check runs on one stream."""
    sc = scenes.make_scene("small", scale=0.5)
    host = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()) if pinned else np.ascontiguousarray

    def create(cams, pts, oc, op, uv, depth):
        return ba.Problem(host(cams), host(pts), host(oc), host(op), host(uv), host(depth))

    args = [sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, sc.obs_uv, sc.depth]
    bad_uv = sc.obs_uv.copy()
    bad_uv[7, 0] = np.nan
    bad_oc = sc.obs_cam.copy()
    bad_oc[3] = sc.spec.n_cams
    for (uv, oc), msg in [((bad_uv, sc.obs_cam), "non-finite observation"),
                          ((sc.obs_uv, bad_oc), "index out of range"),
                          ((bad_uv, bad_oc), "non-finite observation")]:
        with pytest.raises(ba.BAError, match="invalid argument"):
            create(args[0], args[1], oc, args[3], uv, args[5])
        assert msg in ba.lib().ba_last_error().decode()
    # and a valid problem from the same host arrays solves
    p = create(*args)
    p.lm_step()
