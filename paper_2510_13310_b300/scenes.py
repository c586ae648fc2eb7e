"""Seeded synthetic bundle-adjustment scenes.

This module only draws random numbers and synthesises measurements; it holds no
part of the solver (no Jacobians, normal equations, extraction or LM logic).
Both the CUDA path and the CPU oracle are fed from here, and nothing here
imports either of them.

Scene recipe (stands in for the 1DSfM / ScanNet scenes the paper measures on,
which are not available): cameras on a radius-3 circle in the z=0 plane look at
the origin, points are uniform in the unit sphere, every point is seen by a
random subset of cameras, observations carry N(0, sigma_px) pixel noise, a
fraction are replaced by uniform outliers, and a Bernoulli subset carries a
metric depth prior (true camera-frame depth times 1 + N(0, sigma_d)).
The camera is the 9-parameter radial model [axis-angle w, t, f, k1, k2] with
the principal point fixed at the image centre (the paper's Sec. 3.2 uses a
quaternion + centre + focal variant; the 9-parameter form is the one these
workloads are specified in).

The measurement synthesis below projects ground-truth points with the
rotation *matrix* of a look-at frame; the solvers use the axis-angle vector
written out from it, so a zero cost at the ground truth cross-checks both.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial.transform import Rotation

IMG_W, IMG_H = 640, 480
CX, CY = 320.0, 240.0


@dataclasses.dataclass(frozen=True)
class SceneSpec:
    """Shape of one synthetic workload."""
    name: str
    n_cams: int
    n_pts: int
    track_min: int
    track_max: int
    track_mean: float          # mean track length (fixed length when min == max)
    outlier_frac: float = 0.02
    depth_frac: float = 0.5    # fraction of observations with a depth prior
    depth_sigma: float = 0.01  # relative depth-prior noise
    pixel_sigma: float = 0.5
    focal: float = 500.0
    rot_perturb_deg: float = 2.0
    trans_perturb: float = 0.05
    pt_perturb: float = 0.05
    seed: int = 1000


# The five workloads: FP64 small scene, 1M-observation medium scene, 8M-observation
# scene with dynamic extraction, differentiable-BA scene, dense co-visible scene.
SPECS = {
    "small": SceneSpec("small", 20, 2_000, 10, 10, 10.0, seed=1000),
    "medium": SceneSpec("medium", 200, 100_000, 3, 20, 10.0, seed=1001),
    "large": SceneSpec("large", 1_500, 1_000_000, 2, 40, 8.0, outlier_frac=0.05,
                       depth_frac=0.3, depth_sigma=0.03, seed=1002),
    "diff": SceneSpec("diff", 100, 20_000, 10, 10, 10.0, seed=1003),
    "dense": SceneSpec("dense", 2_000, 400_000, 30, 30, 30.0, seed=1004),
    "window": SceneSpec("window", 1_500, 300_000, 3, 12, 6.0, seed=1005),
    # a mid-size scene in the many-runs regime (nearly every camera pair shares a few
    # points): the camera-owned formation with its Y^ rows (134 MB) past L2
    "dense_mid": SceneSpec("dense_mid", 500, 100_000, 12, 12, 12.0, seed=1006),
}
# scenes whose tracks are windows of neighbouring cameras
WINDOWED = {"window"}


@dataclasses.dataclass
class Scene:
    spec: SceneSpec
    cams_gt: np.ndarray   # [C,9] float64
    pts_gt: np.ndarray    # [P,3] float64
    cams0: np.ndarray     # [C,9] float64 initial state
    pts0: np.ndarray      # [P,3] float64 initial state
    obs_cam: np.ndarray   # [N] int32
    obs_pt: np.ndarray    # [N] int32
    obs_uv: np.ndarray    # [N,2] float64 pixels
    depth: np.ndarray     # [N] float64, 0 where no prior
    is_outlier: np.ndarray  # [N] bool
    fixed_cams: np.ndarray  # [F] int32

    @property
    def n_obs(self) -> int:
        return int(self.obs_cam.shape[0])


def _lookat_rotation(centre: np.ndarray) -> np.ndarray:
    """World-to-camera rotation of a camera at `centre` looking at the origin,
    +z forward, +y down, world +z up."""
    fwd = -centre / np.linalg.norm(centre)
    up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    return np.stack([right, down, fwd])


def _truncated_geometric_p(lo: int, hi: int, mean: float) -> float:
    """Success probability p of a geometric law truncated to [lo, hi] whose mean is `mean`."""
    ks = np.arange(lo, hi + 1, dtype=np.float64)

    def m(p):
        w = (1.0 - p) ** (ks - lo)
        return float((ks * w).sum() / w.sum())

    a, b = 1e-9, 1.0 - 1e-9   # m decreases in p
    for _ in range(200):
        c = 0.5 * (a + b)
        if m(c) > mean:
            a = c
        else:
            b = c
    return 0.5 * (a + b)


def _track_lengths(rng, spec: SceneSpec) -> np.ndarray:
    if spec.track_min == spec.track_max:
        return np.full(spec.n_pts, spec.track_min, dtype=np.int64)
    p = _truncated_geometric_p(spec.track_min, spec.track_max, spec.track_mean)
    ks = np.arange(spec.track_min, spec.track_max + 1)
    w = (1.0 - p) ** (ks - spec.track_min)
    return rng.choice(ks, size=spec.n_pts, p=w / w.sum()).astype(np.int64)


def _random_subsets(rng, n_items: int, sizes: np.ndarray) -> list[np.ndarray] | np.ndarray:
    """For each row draw `sizes[i]` distinct items uniformly from range(n_items).

    Uses the first `sizes[i]` distinct values of an i.i.d. uniform sequence,
    which is a uniform random subset; rows that run out are redrawn exactly.
    Returns (flat_items, row_offsets)."""
    n = sizes.shape[0]
    kmax = int(sizes.max())
    extra = 16 if n_items > 4 * kmax else 4 * kmax
    m = kmax + extra
    chunk = max(1, 4_000_000 // m)
    out = np.empty(int(sizes.sum()), dtype=np.int32)
    offs = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        draws = rng.integers(0, n_items, size=(e - s, m))
        order = np.argsort(draws, axis=1, kind="stable")
        srt = np.take_along_axis(draws, order, axis=1)
        first_sorted = np.ones_like(srt, dtype=bool)
        first_sorted[:, 1:] = srt[:, 1:] != srt[:, :-1]
        first = np.empty_like(first_sorted)
        np.put_along_axis(first, order, first_sorted, axis=1)
        rank = np.cumsum(first, axis=1)
        need = sizes[s:e][:, None]
        take = first & (rank <= need)
        ok = take.sum(axis=1) == sizes[s:e]
        for i in range(e - s):
            row = s + i
            if ok[i]:
                out[offs[row]:offs[row + 1]] = draws[i][take[i]]
            else:
                out[offs[row]:offs[row + 1]] = rng.choice(n_items, size=int(sizes[row]), replace=False)
    return out, offs


def project_points(R: np.ndarray, t: np.ndarray, f: np.ndarray, k1: np.ndarray,
                   k2: np.ndarray, X: np.ndarray):
    """Synthesise pixel measurements (radial model, +z forward).  Arrays are per
    observation; R is [N,3,3].  Returns (uv [N,2], camera-frame depth [N])."""
    P = np.einsum("nij,nj->ni", R, X) + t
    xn = P[:, 0] / P[:, 2]
    yn = P[:, 1] / P[:, 2]
    rr = xn * xn + yn * yn
    dist = 1.0 + k1 * rr + k2 * rr * rr
    uv = np.stack([f * dist * xn + CX, f * dist * yn + CY], axis=1)
    return uv, P[:, 2]


def _window_tracks(rng, pts: np.ndarray, C: int, lengths: np.ndarray):
    """Windowed co-visibility: the track of a point takes the `lengths[p]`
    consecutive cameras (on the circle of C) centred on the camera whose azimuth
    is nearest the point's, so cameras i and j share points only when
    |i - j| < max track length (a block-banded reduced camera system)."""
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    centre = np.rint(phi / (2.0 * math.pi) * C).astype(np.int64) % C
    offs = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=offs[1:])
    out = np.empty(int(offs[-1]), dtype=np.int32)
    for L in np.unique(lengths):
        rows = np.flatnonzero(lengths == L)
        start = centre[rows] - (L - 1) // 2
        cams = (start[:, None] + np.arange(L)[None, :]) % C
        # the order inside a track is random, as with drawn subsets
        cams = np.take_along_axis(cams, rng.permuted(np.tile(np.arange(L), (rows.size, 1)), axis=1), axis=1)
        out[(offs[rows][:, None] + np.arange(L)[None, :]).ravel()] = cams.ravel()
    return out, offs


def make_scene(spec: SceneSpec | str, *, seed: int | None = None, noise: bool = True,
               outliers: bool = True, depth_priors: bool = True,
               scale: float | None = None, shuffle: bool = True,
               frustum_exit_frac: float = 0.0, covis: str | None = None,
               camera_model: str = "radial") -> Scene:
    """Generate a seeded scene.

    `noise=False` removes pixel and depth noise, `outliers=False` removes the
    outliers, `depth_priors=False` clears every prior.  `scale` shrinks the
    camera and point counts (for reduced-size parity cases).

    `camera_model` "centre" gives cameras in the parameterisation of Sec. 3.2
    (centre, rotation, focal length, no distortion) in the nine slots
    [w, c, f, 0, 0]: measurements synthesised with k1 = k2 = 0, the start moves
    each centre by trans_perturb * |c| in a random direction.

    `covis` chooses the cameras of each track: "random" (distinct cameras drawn
    uniformly) or "window" (the angularly nearest cameras; the default for the
    scenes in WINDOWED).

    `frustum_exit_frac` injects frustum exits: that fraction of the points with
    horizontal radius >= 0.5 starts lifted to height 1.35 (+ U(0, 0.1)) above the
    camera plane, which puts it above the image of its nearer cameras (camera-frame
    depth below ~2.8) and inside the image of its farther ones, while its true
    position projects inside every image.  Those observations are invalid at the
    start and valid at the solution.  The draw comes after every other draw, so
    the rest of the scene is the same as without it."""
    if isinstance(spec, str):
        if covis is None:
            covis = "window" if spec in WINDOWED else "random"
        spec = SPECS[spec]
    covis = covis or "random"
    if scale is not None:
        spec = dataclasses.replace(spec, n_cams=max(4, int(round(spec.n_cams * scale))),
                                   n_pts=max(8, int(round(spec.n_pts * scale))))
    if spec.track_max > spec.n_cams:
        spec = dataclasses.replace(spec, track_max=spec.n_cams,
                                   track_min=min(spec.track_min, spec.n_cams),
                                   track_mean=min(spec.track_mean, spec.n_cams))
    rng = np.random.Generator(np.random.PCG64(spec.seed if seed is None else seed))
    C, P = spec.n_cams, spec.n_pts

    # cameras
    phi = 2.0 * math.pi * np.arange(C) / C
    centres = 3.0 * np.stack([np.cos(phi), np.sin(phi), np.zeros(C)], axis=1)
    Rs = np.stack([_lookat_rotation(c) for c in centres])
    ts = -np.einsum("cij,cj->ci", Rs, centres)
    focal = spec.focal * (1.0 + 0.02 * rng.standard_normal(C))
    k1 = 0.01 * rng.standard_normal(C)
    k2 = 0.01 * rng.standard_normal(C)
    centre_model = camera_model == "centre"
    if centre_model:
        k1[:] = 0.0
        k2[:] = 0.0
    cams_gt = np.concatenate([Rotation.from_matrix(Rs).as_rotvec(), centres if centre_model else ts,
                              focal[:, None], k1[:, None], k2[:, None]], axis=1)

    # points uniform in the unit sphere
    pts = np.empty((0, 3))
    while pts.shape[0] < P:
        cand = rng.uniform(-1.0, 1.0, size=(2 * (P - pts.shape[0]) + 16, 3))
        cand = cand[(cand * cand).sum(1) <= 1.0]
        pts = np.concatenate([pts, cand])
    pts_gt = np.ascontiguousarray(pts[:P])

    # tracks
    lengths = _track_lengths(rng, spec)
    if covis == "window":
        cams_flat, offs = _window_tracks(rng, pts_gt, C, lengths)
    else:
        cams_flat, offs = _random_subsets(rng, C, lengths)
    obs_pt = np.repeat(np.arange(P, dtype=np.int32), lengths)
    obs_cam = cams_flat.astype(np.int32)
    N = obs_cam.shape[0]

    uv, z = project_points(Rs[obs_cam], ts[obs_cam], focal[obs_cam], k1[obs_cam],
                           k2[obs_cam], pts_gt[obs_pt])
    if noise:
        uv = uv + spec.pixel_sigma * rng.standard_normal((N, 2))
    is_out = np.zeros(N, dtype=bool)
    if outliers and spec.outlier_frac > 0:
        is_out = rng.random(N) < spec.outlier_frac
        n_out = int(is_out.sum())
        uv[is_out] = np.stack([rng.uniform(0, IMG_W, n_out), rng.uniform(0, IMG_H, n_out)], 1)
    depth = np.zeros(N)
    if depth_priors and spec.depth_frac > 0:
        has = rng.random(N) < spec.depth_frac
        dn = spec.depth_sigma * rng.standard_normal(N) if noise else np.zeros(N)
        depth[has] = z[has] * (1.0 + dn[has])

    # initial state: every non-gauge pose rotated by exactly rot_perturb_deg about a
    # random axis and moved by trans_perturb*|t| in a random direction
    fixed = np.array([0], dtype=np.int32)
    axes = rng.standard_normal((C, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    dirs = rng.standard_normal((C, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rot0 = Rotation.from_rotvec(axes * math.radians(spec.rot_perturb_deg)) * Rotation.from_matrix(Rs)
    base_t = centres if centre_model else ts
    t0 = base_t + spec.trans_perturb * np.linalg.norm(base_t, axis=1, keepdims=True) * dirs
    cams0 = np.concatenate([rot0.as_rotvec(), t0, cams_gt[:, 6:9]], axis=1)
    cams0[fixed] = cams_gt[fixed]
    pts0 = pts_gt + spec.pt_perturb * rng.standard_normal((P, 3))

    if shuffle:
        perm = rng.permutation(N)
    if frustum_exit_frac > 0.0:
        wide = np.flatnonzero(np.hypot(pts_gt[:, 0], pts_gt[:, 1]) >= 0.5)
        lift = wide[rng.random(wide.shape[0]) < frustum_exit_frac]
        pts0[lift, 2] = 1.35 + 0.1 * rng.random(lift.shape[0])

    if shuffle:
        obs_cam, obs_pt, uv, depth, is_out = obs_cam[perm], obs_pt[perm], uv[perm], depth[perm], is_out[perm]

    return Scene(spec, np.ascontiguousarray(cams_gt), pts_gt, np.ascontiguousarray(cams0),
                 np.ascontiguousarray(pts0), np.ascontiguousarray(obs_cam, dtype=np.int32),
                 np.ascontiguousarray(obs_pt, dtype=np.int32), np.ascontiguousarray(uv),
                 np.ascontiguousarray(depth), is_out, fixed)


# ---------------------------------------------------------------------------
# global positioning scenes (Sec. 3.1 / 4.1): rays from known rotations
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class GPScene:
    spec: SceneSpec
    centres_gt: np.ndarray  # [C,3] camera centres
    pts_gt: np.ndarray      # [P,3]
    centres0: np.ndarray    # [C,3] initial state
    pts0: np.ndarray        # [P,3]
    scales0: np.ndarray     # [N] initial scale of every observation (1 / initial range)
    obs_cam: np.ndarray     # [N] int32
    obs_pt: np.ndarray      # [N] int32
    rays: np.ndarray        # [N,3] unit ray from the camera centre toward the feature (world frame)
    depth: np.ndarray       # [N] metric range prior along the ray, 0 where none
    is_outlier: np.ndarray  # [N] bool
    fixed_cams: np.ndarray  # [F] int32

    @property
    def n_obs(self) -> int:
        return int(self.obs_cam.shape[0])


def make_gp_scene(spec: SceneSpec | str, *, seed: int | None = None, noise: bool = True,
                  outliers: bool = True, depth_priors: bool = True,
                  scale: float | None = None) -> GPScene:
    """A global-positioning scene on the same geometry and tracks as make_scene:
    the rays are the true camera-to-point directions (rotations are known in GP),
    perturbed by an angular noise of pixel_sigma / focal radians per axis and
    renormalised; outliers are uniform random directions; a Bernoulli fraction
    `depth_frac` of observations carries a metric range prior
    |X - c| (1 + N(0, depth_sigma)).  Start: centres moved by trans_perturb * 3 in
    a random direction (camera 0, the gauge, kept), points by N(0, pt_perturb),
    every scale 1 / |X0 - c0|."""
    base = make_scene(spec, seed=seed, noise=False, outliers=False, depth_priors=False,
                      scale=scale, shuffle=True)
    spec = base.spec
    rng = np.random.Generator(np.random.PCG64((spec.seed if seed is None else seed) + 7919))
    R = Rotation.from_rotvec(base.cams_gt[:, :3]).as_matrix()
    centres = -np.einsum("cji,cj->ci", R, base.cams_gt[:, 3:6])
    C, P, N = spec.n_cams, spec.n_pts, base.n_obs
    diff = base.pts_gt[base.obs_pt] - centres[base.obs_cam]
    rng_len = np.linalg.norm(diff, axis=1)
    rays = diff / rng_len[:, None]
    if noise:
        rays = rays + (spec.pixel_sigma / spec.focal) * rng.standard_normal((N, 3))
        rays /= np.linalg.norm(rays, axis=1, keepdims=True)
    is_out = np.zeros(N, dtype=bool)
    if outliers and spec.outlier_frac > 0:
        is_out = rng.random(N) < spec.outlier_frac
        r = rng.standard_normal((int(is_out.sum()), 3))
        rays[is_out] = r / np.linalg.norm(r, axis=1, keepdims=True)
    depth = np.zeros(N)
    if depth_priors and spec.depth_frac > 0:
        has = rng.random(N) < spec.depth_frac
        dn = spec.depth_sigma * rng.standard_normal(N) if noise else np.zeros(N)
        depth[has] = rng_len[has] * (1.0 + dn[has])
    fixed = np.array([0], dtype=np.int32)
    dirs = rng.standard_normal((C, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    centres0 = centres + spec.trans_perturb * 3.0 * dirs
    centres0[fixed] = centres[fixed]
    pts0 = base.pts_gt + spec.pt_perturb * rng.standard_normal((P, 3))
    scales0 = 1.0 / np.linalg.norm(pts0[base.obs_pt] - centres0[base.obs_cam], axis=1)
    return GPScene(spec, np.ascontiguousarray(centres), base.pts_gt, np.ascontiguousarray(centres0),
                   np.ascontiguousarray(pts0), np.ascontiguousarray(scales0), base.obs_cam, base.obs_pt,
                   np.ascontiguousarray(rays), np.ascontiguousarray(depth), is_out, fixed)
