"""Seeded synthetic inputs for geometry-aware pairwise matching (arXiv 1512.06235, Sec. 6.2).

This module is shared by the tests, the benchmark and the smoke check.  It holds the *inputs* only -- cameras,
3D points, keypoints, scales, descriptors, the fundamental matrix of each pair and the pair list -- and none of
the method's arithmetic (no epipolar line, band test, descriptor distance or ratio test lives here).

Conventions
-----------
* Pinhole cameras ``x ~ K (R X + t)``; the camera centre is ``C = -R^T t``; image x to the right, y down.
* The fundamental matrix of an ordered pair (A, B) maps a point of A to its epipolar line in B:
  ``l_B = F (x_A, y_A, 1)^T`` and ``x_B^T F x_A = 0``.  From the coplanarity of the two viewing rays and the
  baseline, ``F = K_B^{-T} R_B [C_A - C_B]_x R_A^T K_A^{-1}``.  (Eq. 1 of the paper prints the transposed
  form.)  F is normalised to unit Frobenius norm in FP64 and then rounded to FP32; the FP32 values are the input.
* Descriptors: a uniform [0, 255] base per 3D point; each view adds N(0, 8^2), rounds and clips to [0, 255].
  Distractor keypoints are uniform in the image with uniform descriptors.
* Scales: every 3D point has an intrinsic scale, log-normal(ln 2, 0.5) from a generator of its own (seed ^ 0x5CA1E,
  so that the keypoints and descriptors do not depend on it); a projection's scale is the point's scale times a
  log-normal(0, 0.125) jitter, so the same points are high-scale in every image that sees them (the property the
  coarse stage relies on, Sec. 4).  Distractor scales are log-normal(ln 2, 0.5).
* Keypoint order inside an image is shuffled; ``pid`` keeps the 3D point id (-1 for distractors), which gives
  the known correspondences.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1512_06235
DESC_DIM = 128


@dataclass
class Image:
    width: int
    height: int
    xy: np.ndarray          # float32 [n, 2]
    scale: np.ndarray       # float32 [n]
    desc: np.ndarray        # uint8 [n, 128]
    pid: np.ndarray         # int32 [n], 3D point id or -1

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])


@dataclass
class Pair:
    a: int                  # query image
    b: int                  # target image
    F: np.ndarray           # float32 [9], row-major, l_B = F (x_A, y_A, 1)
    d: float = 4.0          # band half-width in px (max point-to-line distance); inf = whole image
    p: int = 4              # ratio test threshold p/q
    q: int = 5


@dataclass
class Camera:
    K: np.ndarray
    R: np.ndarray
    t: np.ndarray

    @property
    def centre(self) -> np.ndarray:
        return -self.R.T @ self.t


@dataclass
class Scene:
    name: str
    images: list
    pairs: list
    cameras: list = field(default_factory=list)
    info: dict = field(default_factory=dict)


# ---------------------------------------------------------------- geometry helpers (inputs only)

def intrinsics(f: float = 1200.0, w: int = 1600, h: int = 1200) -> np.ndarray:
    return np.array([[f, 0.0, w / 2.0], [0.0, f, h / 2.0], [0.0, 0.0, 1.0]])


def rot_y(deg: float) -> np.ndarray:
    t = math.radians(deg)
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def look_at(centre, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World-to-camera rotation for a camera at ``centre`` looking at ``target`` (image y points down)."""
    f = np.asarray(target, float) - np.asarray(centre, float)
    f /= np.linalg.norm(f)
    x = np.cross(f, np.asarray(up, float))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    return np.stack([x, y, f])


def camera_at(K, R, centre) -> Camera:
    return Camera(K=np.asarray(K, float), R=np.asarray(R, float), t=-np.asarray(R, float) @ np.asarray(centre, float))


def skew(v) -> np.ndarray:
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def fundamental(cam_a: Camera, cam_b: Camera) -> np.ndarray:
    """F with l_B = F x_A, from the two poses (FP64, unit Frobenius norm, then FP32)."""
    F = np.linalg.inv(cam_b.K).T @ cam_b.R @ skew(cam_a.centre - cam_b.centre) @ cam_a.R.T @ np.linalg.inv(cam_a.K)
    F = F / np.linalg.norm(F)
    return F.astype(np.float32).reshape(9)


def project(cam: Camera, X: np.ndarray):
    """Pixel coordinates and depth of world points X [m, 3]."""
    Xc = X @ cam.R.T + cam.t
    z = Xc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        uv = (Xc @ cam.K.T)[:, :2] / z[:, None]
    return uv, z


def inside(uv, w, h):
    return (uv[:, 0] >= 0) & (uv[:, 0] < w) & (uv[:, 1] >= 0) & (uv[:, 1] < h)


def _noisy_in_image(rng, uv, sigma, w, h):
    """Adds N(0, sigma^2) noise; keypoints that leave the image get fresh noise until they are inside."""
    out = uv + rng.normal(0.0, sigma, uv.shape)
    bad = ~inside(out, w, h)
    while bad.any():
        out[bad] = uv[bad] + rng.normal(0.0, sigma, (int(bad.sum()), 2))
        bad = ~inside(out, w, h)
    return out


def _uniform_xy(rng, m, w, h):
    xy = np.stack([rng.uniform(0, w, m), rng.uniform(0, h, m)], axis=1)
    # float32 rounding may land exactly on w or h: keep strictly inside
    xy32 = xy.astype(np.float32)
    xy32[:, 0] = np.minimum(xy32[:, 0], np.nextafter(np.float32(w), np.float32(0)))
    xy32[:, 1] = np.minimum(xy32[:, 1], np.nextafter(np.float32(h), np.float32(0)))
    return xy32


def _view_desc(rng, base_rows, sigma=8.0):
    noisy = np.rint(base_rows.astype(np.float64) + rng.normal(0.0, sigma, base_rows.shape))
    return np.clip(noisy, 0, 255).astype(np.uint8)


def point_scales(seed: int, n_points: int) -> np.ndarray:
    """Intrinsic scale of every 3D point, from a generator independent of the scene's main one."""
    return np.random.default_rng(seed ^ 0x5CA1E).lognormal(math.log(2.0), 0.5, n_points)


def make_image(rng, w, h, uv_true, pids, base, n_distractors, sigma_px=0.5, sigma_desc=8.0,
               point_scale=None) -> Image:
    """One image: noisy projections of the given points plus uniform distractors, in shuffled order."""
    uv = _noisy_in_image(rng, uv_true, sigma_px, w, h).astype(np.float32)
    # keep strictly inside after the float32 rounding
    uv[:, 0] = np.minimum(uv[:, 0], np.nextafter(np.float32(w), np.float32(0)))
    uv[:, 1] = np.minimum(uv[:, 1], np.nextafter(np.float32(h), np.float32(0)))
    dxy = _uniform_xy(rng, n_distractors, w, h)
    xy = np.concatenate([uv, dxy]).astype(np.float32)
    desc = np.concatenate([_view_desc(rng, base[pids], sigma_desc),
                           rng.integers(0, 256, (n_distractors, DESC_DIM), dtype=np.uint8)])
    pid = np.concatenate([pids.astype(np.int32), np.full(n_distractors, -1, np.int32)])
    scale = rng.lognormal(math.log(2.0), 0.5, xy.shape[0])
    if point_scale is not None:   # projections: the point's scale with a small jitter from the same draw
        n_proj = uv.shape[0]
        scale[:n_proj] = point_scale[pids] * (scale[:n_proj] / 2.0) ** 0.25
    scale = scale.astype(np.float32)
    order = rng.permutation(xy.shape[0])
    return Image(width=w, height=h, xy=np.ascontiguousarray(xy[order]), scale=scale[order],
                 desc=np.ascontiguousarray(desc[order]), pid=pid[order])


# ---------------------------------------------------------------- workloads

def two_view(seed: int = SEED_BASE + 1, n_points: int = 1500, n_distractors: int = 500, d: float = 4.0,
             w: int = 1600, h: int = 1200, f: float = 1200.0, baseline_m: float = 1.0, yaw_deg: float = 15.0) -> Scene:
    """Single image pair, plain method: 1500 random 3D points in a 10 m cube centred 15 m in front of camera A;
    camera B 1 m along x and turned 15 deg about y toward the cube; 2000 keypoints per image."""
    rng = np.random.default_rng(seed)
    K = intrinsics(f, w, h)
    cam_a = camera_at(K, np.eye(3), [0.0, 0.0, 0.0])
    cam_b = camera_at(K, rot_y(yaw_deg), [baseline_m, 0.0, 0.0])
    pts = np.zeros((0, 3))
    while pts.shape[0] < n_points:
        X = rng.uniform([-5.0, -5.0, 10.0], [5.0, 5.0, 20.0], (4 * n_points, 3))
        ua, za = project(cam_a, X)
        ub, zb = project(cam_b, X)
        ok = (za > 0) & (zb > 0) & inside(ua, w, h) & inside(ub, w, h)
        pts = np.concatenate([pts, X[ok]])
    pts = pts[:n_points]
    base = rng.integers(0, 256, (n_points, DESC_DIM), dtype=np.uint8)
    pids = np.arange(n_points)
    ps = point_scales(seed, n_points)
    images = [make_image(rng, w, h, project(c, pts)[0], pids, base, n_distractors, point_scale=ps)
              for c in (cam_a, cam_b)]
    pairs = [Pair(0, 1, fundamental(cam_a, cam_b), d)]
    return Scene("two_view_2000", images, pairs, [cam_a, cam_b], {"points": pts})


def facade_points(rng, n_points=50_000, width=40.0, height=15.0, depth=15.0, sigma=0.05):
    """Points on a front plane (z = 0) and two wings (x = -w/2 and x = +w/2, z in [0, depth]), by area, with
    N(0, sigma) noise along each plane's normal.  Returns points and their outward normals (toward z > 0 side)."""
    areas = np.array([width * height, depth * height, depth * height])
    which = rng.choice(3, n_points, p=areas / areas.sum())
    X = np.zeros((n_points, 3))
    N = np.zeros((n_points, 3))
    m0, m1, m2 = which == 0, which == 1, which == 2
    X[m0] = np.stack([rng.uniform(-width / 2, width / 2, m0.sum()), rng.uniform(0, height, m0.sum()),
                      np.zeros(m0.sum())], 1)
    N[m0] = [0.0, 0.0, 1.0]
    for m, sx in ((m1, -1.0), (m2, 1.0)):
        X[m] = np.stack([np.full(m.sum(), sx * width / 2), rng.uniform(0, height, m.sum()),
                         rng.uniform(0, depth, m.sum())], 1)
        N[m] = [-sx, 0.0, 0.0]
    X += N * rng.normal(0.0, sigma, (n_points, 1))
    return X, N


def _select_pairs(vis_sets, n_points, n_pairs, min_covis):
    """Top pairs by co-visible point count (Sec. 6.1 with T = min_covis), unique (a < b)."""
    n = len(vis_sets)
    M = np.zeros((n, n_points), np.float32)
    for i, s in enumerate(vis_sets):
        M[i, s] = 1.0
    C = (M @ M.T).astype(np.int64)
    iu, ju = np.triu_indices(n, 1)
    cnt = C[iu, ju]
    keep = cnt >= min_covis
    iu, ju, cnt = iu[keep], ju[keep], cnt[keep]
    order = np.lexsort((ju, iu, -cnt))[:n_pairs]
    return [(int(iu[k]), int(ju[k]), int(cnt[k])) for k in order]


def facade(seed: int = SEED_BASE + 2, n_images: int = 100, n_kp=8000, proj_frac: float = 0.7,
           n_points: int = 50_000, n_pairs: int = 1200, min_covis: int = 50, d=4.0,
           w: int = 1600, h: int = 1200, f: float = 1200.0, radius: float = 25.0, arc_len: float = 30.0) -> Scene:
    """Small component: cameras on a 30 m arc (radius 25 m, 1.6 m high) looking at a 50k-point facade of three
    planes; ``n_kp`` keypoints per image (an int, or an array of per-image counts), 70 % projections of visible
    points, 30 % distractors; the top ``n_pairs`` pairs with at least ``min_covis`` co-visible keypoints.
    ``d`` is one band for all pairs or a callable ``rng -> d`` drawn per pair."""
    rng = np.random.default_rng(seed)
    X, Nrm = facade_points(rng, n_points)
    K = intrinsics(f, w, h)
    target = np.array([0.0, 7.5, 0.0])
    phis = np.linspace(-arc_len / radius / 2, arc_len / radius / 2, n_images)
    cams = [camera_at(K, look_at([radius * math.sin(p), 1.6, radius * math.cos(p)], target),
                      [radius * math.sin(p), 1.6, radius * math.cos(p)]) for p in phis]
    base = rng.integers(0, 256, (n_points, DESC_DIM), dtype=np.uint8)
    kps = np.broadcast_to(np.asarray(n_kp), (n_images,)).astype(np.int64)
    ps = point_scales(seed, n_points)
    images, vis_sets = [], []
    for ci, cam in enumerate(cams):
        uv, z = project(cam, X)
        facing = np.einsum("ij,ij->i", Nrm, cam.centre[None, :] - X) > 0
        vis = np.nonzero((z > 0.1) & inside(uv, w, h) & facing)[0]
        n_proj = min(int(round(proj_frac * kps[ci])), vis.size)
        sel = np.sort(rng.choice(vis, n_proj, replace=False))
        images.append(make_image(rng, w, h, uv[sel], sel, base, int(kps[ci]) - n_proj, point_scale=ps))
        vis_sets.append(sel)
    chosen = _select_pairs(vis_sets, n_points, n_pairs, min_covis)
    pairs = []
    for a, b, _ in chosen:
        dd = float(d(rng)) if callable(d) else float(d)
        pairs.append(Pair(a, b, fundamental(cams[a], cams[b]), dd))
    return Scene(f"facade_{n_images}x{int(kps.mean())}", images, pairs, cams,
                 {"covis": [c for _, _, c in chosen]})


def street(seed: int = SEED_BASE + 3, n_images: int = 1000, n_points: int = 1_000_000, n_kp=None,
           kp_range=(2000, 20000), n_pairs: int = 20_000, min_covis: int = 50, d=None, proj_frac: float = 0.7,
           w: int = 1600, h: int = 1200, f: float = 1200.0, spacing: float = 0.5) -> Scene:
    """Street-like component: two facades at x = -10 m and x = +10 m along a 500 m path (points 0-20 m high),
    cameras every 0.5 m on the path at 1.6 m, alternately looking at the left and the right facade (turned
    30 deg forward); per-image keypoint counts log-uniform in ``kp_range`` unless ``n_kp`` is given; band
    ``d`` per pair uniform in [2, 8] px unless given."""
    rng = np.random.default_rng(seed)
    length = n_images * spacing
    side = rng.integers(0, 2, n_points) * 2 - 1
    X = np.stack([side * 10.0 + rng.normal(0, 0.05, n_points), rng.uniform(0, 20.0, n_points),
                  rng.uniform(-5.0, length + 5.0, n_points)], 1)
    Nrm = np.stack([-side.astype(float), np.zeros(n_points), np.zeros(n_points)], 1)
    K = intrinsics(f, w, h)
    cams = []
    for i in range(n_images):
        c = np.array([0.0, 1.6, i * spacing])
        look_side = 1.0 if i % 2 == 0 else -1.0
        tgt = c + np.array([look_side * 10.0, 3.0, 10.0 * math.tan(math.radians(30.0))])
        cams.append(camera_at(K, look_at(c, tgt), c))
    if n_kp is None:
        kps = np.exp(rng.uniform(math.log(kp_range[0]), math.log(kp_range[1]), n_images)).astype(np.int64)
    else:
        kps = np.broadcast_to(np.asarray(n_kp), (n_images,)).astype(np.int64)
    base = rng.integers(0, 256, (n_points, DESC_DIM), dtype=np.uint8)
    ps = point_scales(seed, n_points)
    images, vis_sets = [], []
    order = np.argsort(X[:, 2])
    zs = X[order, 2]
    for ci, cam in enumerate(cams):
        cz = cam.centre[2]
        lo, hi = np.searchsorted(zs, cz - 5.0), np.searchsorted(zs, cz + 60.0)
        cand = order[lo:hi]
        uv, z = project(cam, X[cand])
        facing = np.einsum("ij,ij->i", Nrm[cand], cam.centre[None, :] - X[cand]) > 0
        ok = (z > 0.1) & inside(uv, w, h) & facing
        vis = cand[ok]
        uv = uv[ok]
        n_proj = min(int(round(proj_frac * kps[ci])), vis.size)
        pick = np.sort(rng.choice(vis.size, n_proj, replace=False))
        sel = vis[pick]
        images.append(make_image(rng, w, h, uv[pick], sel, base, int(kps[ci]) - n_proj, point_scale=ps))
        vis_sets.append(sel)
    chosen = _select_pairs_sparse(vis_sets, n_pairs, min_covis)
    pairs = []
    for a, b, _ in chosen:
        dd = float(rng.uniform(2.0, 8.0)) if d is None else (float(d(rng)) if callable(d) else float(d))
        pairs.append(Pair(a, b, fundamental(cams[a], cams[b]), dd))
    return Scene(f"street_{n_images}", images, pairs, cams, {"covis": [c for _, _, c in chosen]})


def _select_pairs_sparse(vis_sets, n_pairs, min_covis):
    """Co-visibility counts through a sparse point->camera incidence (scipy), top pairs with count >= T."""
    import scipy.sparse as sp
    rows = np.concatenate([np.full(s.size, i, np.int64) for i, s in enumerate(vis_sets)])
    cols = np.concatenate(vis_sets).astype(np.int64)
    uniq, cols_c = np.unique(cols, return_inverse=True)
    M = sp.csr_matrix((np.ones(rows.size, np.float32), (rows, cols_c)), shape=(len(vis_sets), uniq.size))
    C = (M @ M.T).tocoo()
    keep = (C.row < C.col) & (C.data >= min_covis)
    r, c, v = C.row[keep], C.col[keep], C.data[keep].astype(np.int64)
    order = np.lexsort((c, r, -v))[:n_pairs]
    return [(int(r[k]), int(c[k]), int(v[k])) for k in order]


# ---------------------------------------------------------------- tiny synthetic inputs for unit tests

def random_small(seed: int, n_a: int, n_b: int, w: int = 320, h: int = 240, d: float = 4.0,
                 desc_levels: int = 256) -> Scene:
    """Two random cameras (generic relative pose) over random points, with a few keypoints per image.
    ``desc_levels`` < 256 draws descriptors from a small alphabet, which makes equal distances (ties) common."""
    rng = np.random.default_rng(seed)
    K = intrinsics(0.75 * w, w, h)
    cam_a = camera_at(K, np.eye(3), [0.0, 0.0, 0.0])
    yaw = rng.uniform(-20, 20)
    cb = rng.normal(0, 1.0, 3) * [1.0, 0.3, 0.3]
    cam_b = camera_at(K, rot_y(yaw) @ _rot_x(rng.uniform(-5, 5)), cb)
    F = fundamental(cam_a, cam_b)
    xyA = _uniform_xy(rng, n_a, w, h)
    xyB = _uniform_xy(rng, n_b, w, h)
    step = 256 // desc_levels
    dA = (rng.integers(0, desc_levels, (n_a, DESC_DIM)) * step).astype(np.uint8)
    dB = (rng.integers(0, desc_levels, (n_b, DESC_DIM)) * step).astype(np.uint8)
    ims = [Image(w, h, xyA, np.ones(n_a, np.float32), dA, np.full(n_a, -1, np.int32)),
           Image(w, h, xyB, np.ones(n_b, np.float32), dB, np.full(n_b, -1, np.int32))]
    return Scene(f"random_small_{seed}", ims, [Pair(0, 1, F, d)], [cam_a, cam_b])


def _rot_x(deg: float) -> np.ndarray:
    t = math.radians(deg)
    c, s = math.cos(t), math.sin(t)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


RECTIFIED_F = np.array([0, 0, 0, 0, 0, -1, 0, 1, 0], np.float32)
"""F of a rectified pair (pure translation along x, equal intrinsics): l_B = (0, -1, y_A), i.e. y' = y."""


def visibility(scene):
    """Point -> camera CSR of a scene (the coarse model's point-camera visibility, Sec. 6.1): point p is seen by
    camera c iff one of c's keypoints projects p.  Returns (point_off int64 [P+1], point_cams int32, n_cams); only
    points seen by at least one camera are listed."""
    n_cams = len(scene.images)
    cams, pts = [], []
    for c, im in enumerate(scene.images):
        pid = np.unique(im.pid[im.pid >= 0])
        cams.append(np.full(pid.size, c, np.int64))
        pts.append(pid.astype(np.int64))
    cams = np.concatenate(cams)
    pts = np.concatenate(pts)
    order = np.lexsort((cams, pts))
    cams, pts = cams[order], pts[order]
    _, start = np.unique(pts, return_index=True)
    point_off = np.append(start, pts.size).astype(np.int64)
    return point_off, cams.astype(np.int32), n_cams


def path_visibility(n_cams: int, n_points: int, seed: int = SEED_BASE + 6):
    """Point -> camera CSR of a long image sequence (the coarse model's visibility of a street or a corridor, Sec.
    6.1): every point is seen by a run of 2-14 consecutive cameras from a random start (wrapping at the end), and 2 %
    of the points also by two cameras half the sequence away.  Returns (point_off int64 [P+1], point_cams int32,
    n_cams); each point's cameras are distinct and ascending."""
    rng = np.random.default_rng(seed)
    start = rng.integers(0, n_cams, n_points)
    deg = rng.integers(2, 15, n_points)
    far = rng.random(n_points) < 0.02
    cols = np.arange(16)
    cam = (start[:, None] + cols[None, :14]) % n_cams
    cam = np.concatenate([cam, (start[:, None] + n_cams // 2 + cols[None, :2]) % n_cams], 1)
    keep = np.concatenate([cols[None, :14] < deg[:, None], np.repeat(far[:, None], 2, 1)], 1)
    cam = np.where(keep, cam, np.iinfo(np.int64).max)
    cam.sort(axis=1)
    n = keep.sum(1)
    off = np.zeros(n_points + 1, np.int64)
    off[1:] = np.cumsum(n)
    return off, cam[cam != np.iinfo(np.int64).max].astype(np.int32), n_cams
