"""ba_create's observation layout, built on the device, against the host
reference builder (whose arrays tests/test_layout_cpu.py checks against
brute-force definitions): point and camera orders, offsets, tile descriptors and
records, camera chunks, the structure hash and the co-visibility runs must be
identical bit for bit, and invalid inputs must be rejected alike."""
import numpy as np
import pytest

from paper_2510_13310_b300 import ba, scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def random_obs(C, P, max_track, seed):
    """Each point seen by a random set of distinct cameras, in shuffled input order."""
    rng = np.random.default_rng(seed)
    oc, op = [], []
    for p in range(P):
        t = int(rng.integers(0, min(max_track, C) + 1))
        cams = rng.choice(C, size=t, replace=False)
        oc.extend(cams.tolist())
        op.extend([p] * t)
    perm = rng.permutation(len(oc))
    oc = np.asarray(oc, np.int32)[perm] if oc else np.zeros(0, np.int32)
    op = np.asarray(op, np.int32)[perm] if op else np.zeros(0, np.int32)
    cams = np.full((C, 9), 0.5)
    pts = np.full((P, 3), 0.25)
    uv = rng.uniform(0, 640, size=(len(oc), 2))
    return cams, pts, oc, op, uv


@pytest.mark.parametrize("C,P,track,seed", [(7, 50, 7, 1), (40, 3000, 40, 2), (25, 2000, 3, 3),
                                            (300, 400, 12, 4), (5, 0, 0, 5), (5, 10, 0, 6),
                                            (2, 70000, 2, 7), (600, 3000, 256, 8)])
def test_device_layout_matches_host_reference(C, P, track, seed):
    assert ba.selftest_layout(*random_obs(C, P, track, seed)) == 0


@pytest.mark.parametrize("name", ["medium", "large"])
def test_device_layout_of_the_workloads(name):
    sc = scenes.make_scene(name)
    assert ba.selftest_layout(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, sc.obs_uv) == 0


def test_invalid_inputs_rejected_alike():
    cams, pts, oc, op, uv = random_obs(6, 40, 5, 11)
    cases = []
    cases.append((cams, pts, np.append(oc, oc[3]), np.append(op, op[3]), np.vstack([uv, uv[:1]]), "duplicate"))
    bad = op.copy()
    bad[7] = 40
    cases.append((cams, pts, oc, bad, uv, "out of range"))
    nan_uv = uv.copy()
    nan_uv[2, 1] = np.nan
    cases.append((cams, pts, oc, op, nan_uv, "non-finite observation"))
    nan_c = cams.copy()
    nan_c[1, 4] = np.inf
    cases.append((nan_c, pts, oc, op, uv, "non-finite camera"))
    long_oc = np.arange(300, dtype=np.int32)[:257]
    cases.append((np.full((300, 9), 0.5), np.full((2, 3), 0.1), long_oc, np.ones(257, np.int32),
                  np.ones((257, 2)), "limit 256"))
    for c, p, o1, o2, u, msg in cases:
        assert ba.selftest_layout(c, p, o1, o2, u) == 0, msg
        with pytest.raises(ba.BAError) as ei:
            ba.Problem(c, p, o1, o2, u, np.zeros(len(o1)))
        assert msg in str(ei.value), (msg, str(ei.value))
