"""Pins of the candidate-pair oracle (Sec. 6.1) against brute force on sets and closed forms (CPU)."""
import itertools

import numpy as np
import pytest

from oracle import pairs as op


def _random_visibility(rng, n_cams, n_points, max_deg):
    off, cams = [0], []
    for _ in range(n_points):
        d = int(rng.integers(0, max_deg + 1))
        cams.extend(sorted(rng.choice(n_cams, min(d, n_cams), replace=False).tolist()))
        off.append(len(cams))
    return np.array(off, np.int64), np.array(cams, np.int32)


def _brute(n_cams, off, cams, T, k):
    """The definition on Python sets: Points(C_i), intersections, ranking, union."""
    points = [set() for _ in range(n_cams)]
    for p in range(len(off) - 1):
        for c in cams[off[p]:off[p + 1]]:
            points[int(c)].add(p)
    chosen = {}
    for q in range(n_cams):
        s = [(len(points[q] & points[i]), i) for i in range(n_cams) if i != q]
        s = [t for t in s if t[0] > T]
        s.sort(key=lambda t: (-t[0], t[1]))
        for cnt, i in s[:k]:
            chosen[(min(q, i), max(q, i))] = cnt
    return np.array([(a, b, c) for (a, b), c in sorted(chosen.items())], np.int64).reshape(-1, 3)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("T,k", [(0, 2), (2, 3), (-1, 100), (5, 1)])
def test_select_pairs_brute_force(seed, T, k):
    rng = np.random.default_rng(seed)
    n_cams = int(rng.integers(3, 12))
    off, cams = _random_visibility(rng, n_cams, int(rng.integers(10, 80)), 5)
    np.testing.assert_array_equal(op.select_pairs(n_cams, off, cams, T, k), _brute(n_cams, off, cams, T, k))


def test_all_points_seen_by_all_cameras():
    """Every count equals the number of points; with k images per query the lowest indices win the ties."""
    n_cams, n_points, k = 7, 20, 2
    off = np.arange(n_points + 1, dtype=np.int64) * n_cams
    cams = np.tile(np.arange(n_cams, dtype=np.int32), n_points)
    got = op.select_pairs(n_cams, off, cams, 8, k)
    want = set()
    for q in range(n_cams):
        others = [i for i in range(n_cams) if i != q][:k]
        want |= {(min(q, i), max(q, i)) for i in others}
    assert [tuple(r[:2]) for r in got] == sorted(want)
    assert (got[:, 2] == n_points).all()
    assert op.select_pairs(n_cams, off, cams, n_points, k).shape == (0, 3)   # > T is strict


def test_covisibility_symmetric_with_degrees_on_diagonal():
    rng = np.random.default_rng(11)
    off, cams = _random_visibility(rng, 9, 200, 6)
    C = op.covisibility(9, off, cams)
    np.testing.assert_array_equal(C, C.T)
    np.testing.assert_array_equal(np.diag(C), np.bincount(cams, minlength=9))
    for i, j in itertools.combinations(range(9), 2):
        pts_i = {p for p in range(len(off) - 1) if i in cams[off[p]:off[p + 1]]}
        pts_j = {p for p in range(len(off) - 1) if j in cams[off[p]:off[p + 1]]}
        assert C[i, j] == len(pts_i & pts_j)


def test_duplicate_camera_rejected():
    with pytest.raises(ValueError):
        op.select_pairs(3, np.array([0, 2]), np.array([1, 1], np.int32), 0, 2)
