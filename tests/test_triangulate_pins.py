"""Pins of the triangulation oracle: exact recovery from noise-free projections, a hand-solved two-view case,
track assembly from labels (CPU)."""
import numpy as np
import pytest

import scenes
from oracle import triangulate as otr


def test_noise_free_projections_recover_the_point(two_view_scene):
    sc = two_view_scene
    Ps = [otr.camera_matrix(c) for c in sc.cameras]
    rng = np.random.default_rng(0)
    X = rng.uniform([-3, -3, 12], [3, 3, 18], (50, 3))
    for Xi in X:
        xy = [scenes.project(c, Xi[None])[0][0] for c in sc.cameras]
        np.testing.assert_allclose(otr.triangulate(Ps, xy), Xi, rtol=1e-9, atol=1e-9)


def test_two_view_by_hand():
    """Cameras at the origin and at x = 1 looking down z (K = I): the point (0.5, 0.25, 2) projects to
    (0.25, 0.125) and (-0.25, 0.125); the equations reduce to x = 0.25 Z, x - 1 = -0.25 Z, y = 0.125 Z."""
    P0 = np.hstack([np.eye(3), np.zeros((3, 1))])
    P1 = np.hstack([np.eye(3), np.array([[-1.0], [0.0], [0.0]])])
    X = otr.triangulate([P0, P1], [(0.25, 0.125), (-0.25, 0.125)])
    np.testing.assert_allclose(X, [0.5, 0.25, 2.0], rtol=0, atol=1e-12)


def test_tracks_from_labels():
    P0 = np.hstack([np.eye(3), np.zeros((3, 1))])
    P1 = np.hstack([np.eye(3), np.array([[-1.0], [0.0], [0.0]])])
    xy0 = np.array([[0.25, 0.125], [9.0, 9.0]])
    xy1 = np.array([[7.0, 7.0], [-0.25, 0.125]])
    labels = np.array([0, 1, 2, 0])   # node 0 (image 0, feature 0) with node 3 (image 1, feature 1)
    roots, nv, X = otr.triangulate_tracks([P0, P1], [xy0, xy1], labels)
    assert roots.tolist() == [0] and nv.tolist() == [2]
    np.testing.assert_allclose(X[0], [0.5, 0.25, 2.0], atol=1e-12)
    # a single observation is not a track; one camera twice is singular
    assert np.isnan(otr.triangulate([P0, P0], [(0.25, 0.125), (0.25, 0.125)])).all()


def _noisy_track(seed, n_views=5):
    rng = np.random.default_rng(seed)
    K = scenes.intrinsics(900.0, 1280, 960)
    cams = []
    for k in range(n_views):
        c = np.array([1.5 * k - 3.0, 0.2 * k, -10.0 + 0.5 * k])
        cams.append(scenes.camera_at(K, scenes.look_at(c, [0.0, 0.0, 0.0]), c))
    Xt = rng.uniform(-1.0, 1.0, 3)
    xy = [scenes.project(c, Xt[None])[0][0] + rng.normal(0.0, 1.5, 2) for c in cams]
    return cams, xy


def _weighted_reprojection(cams, xy, X):
    """sum over views of (depth * |observed - projected|)^2: the algebraic residual of the two rows per view
    written through the camera's projection (x P3 - P1) X = depth * (x - u), with depth = P3 X."""
    f = 0.0
    for c, o in zip(cams, xy):
        uv, z = scenes.project(c, X[None])
        f += (z[0] * np.linalg.norm(np.asarray(o) - uv[0])) ** 2
    return f


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_least_squares_optimality_under_noise(seed):
    """With noisy pixels the point minimises the depth-weighted reprojection error: every small step away from it
    raises the objective, and the objective's central-difference gradient vanishes."""
    cams, xy = _noisy_track(seed)
    X = otr.triangulate([otr.camera_matrix(c) for c in cams], xy)
    f0 = _weighted_reprojection(cams, xy, X)
    rng = np.random.default_rng(seed + 100)
    for _ in range(20):
        step = rng.normal(size=3) * 1e-3
        assert _weighted_reprojection(cams, xy, X + step) > f0
    h = 1e-4
    grad = [(_weighted_reprojection(cams, xy, X + h * e) - _weighted_reprojection(cams, xy, X - h * e)) / (2 * h)
            for e in np.eye(3)]
    curv = (_weighted_reprojection(cams, xy, X + h * np.ones(3)) - f0) / h ** 2
    assert np.abs(grad).max() < 1e-6 * max(curv, 1.0)


def test_affine_change_of_world_frame():
    """An affine change of the world frame X -> H X (rotation, scale, translation) maps cameras to P H^-1 and the
    least-squares point to H X, noise or not."""
    cams, xy = _noisy_track(7)
    Ps = [otr.camera_matrix(c) for c in cams]
    H = np.eye(4)
    H[:3, :3] = 2.5 * scenes.rot_y(30.0)
    H[:3, 3] = [4.0, -1.0, 0.5]
    X = otr.triangulate(Ps, xy)
    Xh = otr.triangulate([P @ np.linalg.inv(H) for P in Ps], xy)
    np.testing.assert_allclose(Xh, H[:3, :3] @ X + H[:3, 3], rtol=1e-9, atol=1e-9)


# ---- per-image tracks (Sec. 6.3: tracks of each query image from its matches in all its candidate images)

def _three_cameras():
    """K = I cameras at the origin, at x = 1 and at y = 1, looking down z."""
    P0 = np.hstack([np.eye(3), np.zeros((3, 1))])
    P1 = np.hstack([np.eye(3), np.array([[-1.0], [0.0], [0.0]])])
    P2 = np.hstack([np.eye(3), np.array([[0.0], [-1.0], [0.0]])])
    return [P0, P1, P2]


def test_image_tracks_by_hand():
    """The point (0.5, 0.25, 2) projects to (0.25, 0.125), (-0.25, 0.125) and (0.25, -0.375).  Image 0 holds it as
    feature 0, image 1 as feature 1, image 2 as feature 0 (the other features are unrelated).  Pairs (0, 1) and
    (0, 2) give image 0's feature 0 a track of three views; pair (1, 2) gives image 1's feature 1 a track of two;
    nodes are image-major (image 1 starts at node 2), so the tracks are nodes 0 and 3."""
    Ps = _three_cameras()
    xy = [np.array([[0.25, 0.125], [5.0, 5.0]]), np.array([[7.0, 7.0], [-0.25, 0.125]]),
          np.array([[0.25, -0.375], [3.0, 1.0]])]
    pairs = [(0, 1), (0, 2), (1, 2)]
    matches = [np.array([[0, 1]]), np.array([[0, 0]]), np.array([[1, 0]])]
    nodes, nv, X = otr.image_tracks(Ps, xy, pairs, matches)
    assert nodes.tolist() == [0, 3] and nv.tolist() == [3, 2]
    np.testing.assert_allclose(X, [[0.5, 0.25, 2.0], [0.5, 0.25, 2.0]], rtol=0, atol=1e-12)
    # a feature without matches forms no track; an empty match list gives no tracks at all
    nodes, nv, X = otr.image_tracks(Ps, xy, pairs, [np.zeros((0, 2), int)] * 3)
    assert nodes.size == 0 and nv.size == 0 and X.shape == (0, 3)


def _noise_free_views(seed, n_cams=5, n_points=40):
    """Noise-free projections of random points into n_cams cameras around them; features of each image in a
    shuffled order; returns cameras, the images' xy, the feature -> point map of each image and the points."""
    rng = np.random.default_rng(seed)
    K = scenes.intrinsics(900.0, 1280, 960)
    cams = []
    for k in range(n_cams):
        c = np.array([2.0 * k - 4.0, 0.3 * k, -12.0])
        cams.append(scenes.camera_at(K, scenes.look_at(c, [0.0, 0.0, 0.0]), c))
    Xw = rng.uniform(-2.0, 2.0, (n_points, 3))
    xy, pid = [], []
    for c in cams:
        order = rng.permutation(n_points)[: n_points - 5]   # every image misses five of the points
        xy.append(scenes.project(c, Xw[order])[0])
        pid.append(order)
    return cams, xy, pid, Xw


def test_image_tracks_noise_free_recover_the_points():
    """Pairs (a, b) for every ordered a != b, matches = the true correspondences: every per-image track comes back
    at its point, and its view count is 1 + the number of other images that see the point."""
    cams, xy, pid, Xw = _noise_free_views(11)
    n = len(cams)
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b]
    matches = []
    for a, b in pairs:
        where_b = {int(p): j for j, p in enumerate(pid[b])}
        matches.append(np.array([[i, where_b[int(p)]] for i, p in enumerate(pid[a]) if int(p) in where_b]))
    nodes, nv, X = otr.image_tracks([otr.camera_matrix(c) for c in cams], xy, pairs, matches)
    base = np.concatenate([[0], np.cumsum([len(x) for x in xy])])
    seen = np.zeros(len(Xw), int)
    for p in pid:
        seen[p] += 1
    assert nodes.size == sum(len(p) for p in pid)   # every feature of every image sees its point at least twice
    for v, m, x in zip(nodes, nv, X):
        k = int(np.searchsorted(base, v, side="right") - 1)
        point = pid[k][v - base[k]]
        assert m == seen[point]
        np.testing.assert_allclose(x, Xw[point], rtol=1e-9, atol=1e-9)


def test_image_tracks_reverse_pairs_duplicate_the_point():
    """Sec. 6.3: a feature pair matched in both directions, (a, i) -> (b, j) and (b, j) -> (a, i), is triangulated
    for image a and again for image b: the same point twice (up to the order of two equal sums)."""
    cams, xy, pid, Xw = _noise_free_views(12, n_cams=2)
    rng = np.random.default_rng(5)
    Ps = [otr.camera_matrix(c) for c in cams]
    noisy = [x + rng.normal(0.0, 1.0, x.shape) for x in xy]
    where_1 = {int(p): j for j, p in enumerate(pid[1])}
    m01 = np.array([[i, where_1[int(p)]] for i, p in enumerate(pid[0]) if int(p) in where_1])
    m10 = m01[:, ::-1][np.argsort(m01[:, 1])]
    nodes, nv, X = otr.image_tracks(Ps, noisy, [(0, 1), (1, 0)], [m01, m10])
    n0 = len(xy[0])
    by_node = dict(zip(nodes.tolist(), X))
    assert (nv == 2).all() and len(nodes) == 2 * len(m01)
    for i, j in m01:
        np.testing.assert_allclose(by_node[int(i)], by_node[n0 + int(j)], rtol=1e-12, atol=1e-12)


def test_image_tracks_merge_into_the_match_components():
    """Merging the per-image tracks (any two tracks sharing an observation are joined) gives the connected
    components of the match graph: the tracks cover every matched node, and a track never spans two components."""
    from oracle import tracks as otk
    rng = np.random.default_rng(4)
    counts = [30, 25, 40, 35]
    pairs = [(0, 1), (0, 2), (1, 2), (2, 3), (3, 0), (1, 0)]
    matches = []
    for a, b in pairs:
        i = np.sort(rng.choice(counts[a], 12, replace=False))
        matches.append(np.stack([i, rng.integers(0, counts[b], 12)], 1))
    base = np.concatenate([[0], np.cumsum(counts)])
    edges = np.concatenate([np.stack([base[a] + m[:, 0], base[b] + m[:, 1]], 1) for (a, b), m in zip(pairs, matches)])
    labels = otk.labels(int(base[-1]), edges)
    xy = [rng.uniform(0, 100, (n, 2)) for n in counts]
    Ps = _three_cameras() + [np.hstack([np.eye(3), np.array([[1.0], [1.0], [0.0]])])]
    nodes, nv, _ = otr.image_tracks(Ps, xy, pairs, matches)
    members = {}
    for (a, b), m in zip(pairs, matches):
        for i, j in m:
            members.setdefault(int(base[a] + i), {int(base[a] + i)}).add(int(base[b] + j))
    assert sorted(members) == nodes.tolist()
    assert [len(members[v]) for v in nodes] == [int(x) for x in nv]   # distinct pairs: distinct observations
    track_edges = np.array([[v, u] for v in nodes for u in members[int(v)] if u != v], np.int64)
    np.testing.assert_array_equal(otk.labels(int(base[-1]), track_edges), labels)
