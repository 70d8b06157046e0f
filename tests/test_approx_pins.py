"""Pins of the approximate-matching oracle (Sec. 6.2.1-6.2.2, App. A): cell geometry by closed forms, chords and
groups of a rectified pair, coverage / containment of C' checked in FP64 geometry, and the 2-NN step against a
pure-Python search (CPU)."""
import math

import numpy as np
import pytest

from oracle import approx as oa

RECTIFIED = np.array([0, 0, 0, 0, 0, -1, 0, 1, 0], np.float32)   # l = (0, -1, y): the horizontal line y' = y


def test_centre_most_cell_closed_forms():
    h = 4.0
    # a point at a cell centre of each grid picks that grid (distance 0)
    for (x, y), g in [((h, h), 0), ((2 * h, h), 1), ((h, 2 * h), 2), ((2 * h, 2 * h), 3), ((5 * h, 7 * h), 0)]:
        c = oa.chosen_cells(np.array([x], np.float32), np.array([y], np.float32), h)[0]
        assert c[0] == g
        ox, oy = (g & 1) * h, (g >> 1) * h
        assert ox + (2 * c[1] + 1) * h == x and oy + (2 * c[2] + 1) * h == y
    # the chosen centre is within h/2 of the point in each axis, and the point lies inside the chosen cell
    rng = np.random.default_rng(0)
    xs, ys = rng.uniform(0, 200, 2000).astype(np.float32), rng.uniform(0, 100, 2000).astype(np.float32)
    for (g, i, j), x, y in zip(oa.chosen_cells(xs, ys, h).tolist(), xs, ys):
        cx, cy = (g & 1) * h + (2 * i + 1) * h, (g >> 1) * h + (2 * j + 1) * h
        assert abs(x - cx) <= h / 2 + 1e-4 and abs(y - cy) <= h / 2 + 1e-4


def test_chords():
    W, H = 100.0, 50.0
    # horizontal line y' = 20: right end (W, 20) at t = W + 20, left end (0, 20) at t = 2W + 2H - 20
    e = oa.chord(*oa.line32(RECTIFIED, 7.0, 20.0), W, H)
    assert (float(e[0][0]), float(e[0][1]), float(e[0][2])) == (W, 20.0, W + 20.0)
    assert (float(e[1][0]), float(e[1][1]), float(e[1][2])) == (0.0, 20.0, 2 * W + 2 * H - 20.0)
    # vertical line x' = 5: (5, 0) at t = 5 and (5, H) at t = 2W + H - 5
    e = oa.chord(np.float32(1.0), np.float32(0.0), np.float32(-5.0), W, H)
    assert [float(v) for v in e[0]] == [5.0, 0.0, 5.0] and [float(v) for v in e[1]] == [5.0, H, 2 * W + H - 5]
    # the diagonal through two corners, and a line that misses the image
    e = oa.chord(np.float32(H), np.float32(-W), np.float32(0.0), W, H)
    assert float(e[0][2]) == 0.0 and float(e[1][2]) == W + H
    assert oa.chord(np.float32(0.0), np.float32(1.0), np.float32(10.0), W, H) is None
    assert oa.chord(np.float32(0.0), np.float32(0.0), np.float32(1.0), W, H) is None


def test_groups_of_a_rectified_pair():
    ys = [30.0, 10.0, 20.5, 13.0, 11.5, 20.0, 500.0]    # the last line misses B (H = 100)
    xy = np.stack([np.full(len(ys), 3.0), ys], 1).astype(np.float32)
    gs, _ = oa.groups(RECTIFIED, xy, 120.0, 100.0)
    # sorted by t1 = W + y: 10 leads 11.5 (1.5 px) but not 13 (3 px); 20 leads 20.5; 30 alone; the lineless one last
    assert gs == [[1, 4], [3], [5, 2], [0], [6]]


def _segment_distance(q, a, b):
    ab = b - a
    L2 = float(ab @ ab)
    t = 0.0 if L2 == 0 else min(1.0, max(0.0, float((q - a) @ ab) / L2))
    return float(np.linalg.norm(q - (a + t * ab)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_candidate_set_coverage_and_containment(seed):
    """C' holds every point of B within h/2 of a sample point (Euclidean) and nothing farther than 3h/2 from one
    (Chebyshev), with the samples recomputed in FP64 from an FP64 chord."""
    rng = np.random.default_rng(seed)
    W, H, h = 320.0, 240.0, 4.0
    xyB = np.stack([rng.uniform(0, W, 6000), rng.uniform(0, H, 6000)], 1).astype(np.float32)
    binned = oa.bins(xyB, h)
    for _ in range(10):
        a, b = rng.normal(size=2)
        c = -(a * rng.uniform(0, W) + b * rng.uniform(0, H))
        a, b, c = np.float32(a), np.float32(b), np.float32(c)
        ends = oa.chord(a, b, c, W, H)
        C = set(oa.candidate_set(ends, h, binned).tolist())
        # FP64 chord and samples
        A = np.array([float(ends[0][0]), float(ends[0][1])])
        B = np.array([float(ends[1][0]), float(ends[1][1])])
        K = math.ceil(np.linalg.norm(B - A) / h)
        S = np.array([(k * A + (K - k) * B) / K for k in range(K + 1)]) if K else A[None]
        P = xyB.astype(np.float64)
        dist = np.sqrt(((P[:, None, :] - S[None, :, :]) ** 2).sum(2)).min(1)
        cheb = np.abs(P[:, None, :] - S[None, :, :]).max(2).min(1)
        must = set(np.nonzero(dist <= h / 2 - 1e-2)[0].tolist())
        may = set(np.nonzero(cheb <= 1.5 * h + 1e-2)[0].tolist())
        assert must <= C <= may
        assert len(C) < len(may) or len(may) == len(must)   # strictly thinner than the containment bound
        # every point of C' is also close to the line
        for pidx in list(C)[:50]:
            assert _segment_distance(P[pidx], A, B) <= 1.5 * h * math.sqrt(2) + 1e-2


def test_matching_against_brute_force():
    rng = np.random.default_rng(5)
    W, H = 160.0, 120.0
    nA, nB = 150, 400
    base = rng.integers(0, 256, (60, 128))
    xyA = np.stack([rng.uniform(0, W, nA), rng.uniform(0, H, nA)], 1).astype(np.float32)
    xyB = np.stack([rng.uniform(0, W, nB), rng.uniform(0, H, nB)], 1).astype(np.float32)
    dA = np.clip(base[rng.integers(0, 60, nA)] + rng.normal(0, 5, (nA, 128)), 0, 255).astype(np.uint8)
    dB = np.clip(base[rng.integers(0, 60, nB)] + rng.normal(0, 5, (nB, 128)), 0, 255).astype(np.uint8)
    F = np.array([0.001, 0.01, -0.5, -0.01, 0.002, -0.8, 0.4, 1.0, -30.0], np.float32)
    for scale in (1.0, 2.5):
        mj = oa.match_pair(xyA, dA, xyB, dB, W, H, F, 4.0, 4, 5, scale)
        h = np.float32(np.float32(4.0) * np.float32(scale))
        gs, ends = oa.groups(F, xyA, W, H)
        binned = oa.bins(xyB, h)
        want = np.full(nA, -1)
        for grp in gs:
            C = oa.candidate_set(ends[grp[0]], h, binned).tolist()
            for qi in grp:
                D = sorted((int(((dA[qi].astype(int) - dB[j].astype(int)) ** 2).sum()), j) for j in C)
                if len(D) >= 2 and 25 * D[0][0] < 16 * D[1][0]:
                    want[qi] = D[0][1]
        np.testing.assert_array_equal(mj, want)
        assert (mj >= 0).sum() > 10
