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
