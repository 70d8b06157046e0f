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
