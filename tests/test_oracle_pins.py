"""Pins of the CPU oracle against things other than itself (CPU only).

* exhaustive matching (d = inf) against scipy's cdist and an int64 brute force (Sec. 2.3 / App. A Step 4);
* hand-derived closed-form band cases (Eqs. 2-3) and ratio-test cases (Sec. 2.3), stored in tests/golden;
* band membership against exact rational arithmetic (Eqs. 2-3, no rounding at all);
* known correspondences of synthetic scenes (recall), and that recall collapses when F is transposed;
* the transpose symmetry of the band for a rectified pair;
* plausibility of |C| / |F_c| against the paper's roughly 1:200 (Sec. 6.2.2);
* the denser-matches effect on repetitive structure (Sec. 6.2.3, Fig. 5).
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
import scenes
from tests import golden


def _exhaustive_reference(dA, dB, p, q):
    """Exhaustive 2-NN + ratio test through scipy's pairwise squared Euclidean distances."""
    nA, nB = dA.shape[0], dB.shape[0]
    out = np.full(nA, -1, np.int64)
    if nB < 2:
        return out
    D = cdist(dA.astype(np.float64), dB.astype(np.float64), "sqeuclidean")
    assert np.all(D == np.rint(D))
    D = D.astype(np.int64)
    for i in range(nA):
        j1 = int(np.argmin(D[i]))                 # first occurrence: lowest index among ties
        d1 = D[i, j1]
        d2 = np.partition(D[i], 1)[1]             # second smallest with multiplicity
        if q * q * d1 < p * p * d2:
            out[i] = j1
    return out


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("levels", [256, 4, 2])
def test_full_band_equals_exhaustive_matching(seed, levels):
    sc = scenes.random_small(seed, 40, 57, desc_levels=levels)
    A, B = sc.images
    for p, q in [(4, 5), (1, 2), (9, 10)]:
        mj, nc = oracle.match_pair(A.xy, A.desc, B.xy, B.desc, sc.pairs[0].F, np.inf, p, q)
        assert nc == A.n * B.n
        np.testing.assert_array_equal(mj, _exhaustive_reference(A.desc, B.desc, p, q))


def test_int64_brute_force_distances():
    rng = np.random.default_rng(7)
    dA = rng.integers(0, 256, (9, 128), dtype=np.uint8)
    dB = rng.integers(0, 256, (11, 128), dtype=np.uint8)
    dA[0] = 255
    dB[0] = 0
    ref = ((dA[:, None, :].astype(np.int64) - dB[None, :, :].astype(np.int64)) ** 2).sum(-1)
    for i in range(9):
        for j in range(11):
            assert oracle.dist2(dA[i], dB[j]) == ref[i, j]
    assert oracle.dist2(dA[0], dB[0]) == 128 * 255 * 255


@pytest.mark.parametrize("case", golden.ratio_cases(), ids=lambda c: c["name"])
def test_ratio_golden(case):
    n = case["bd"].shape[0]
    xyB = np.full((n, 2), 10.0, np.float32).reshape(-1, 2)
    mj, nc = oracle.match_pair(np.array([[5.0, 5.0]], np.float32), case["qd"][None], xyB, case["bd"],
                               np.eye(3, dtype=np.float32).reshape(9), np.inf, case["p"], case["q"])
    assert nc == n
    assert mj[0] == case["expected"]


@pytest.mark.parametrize("case", golden.band_cases(), ids=lambda c: c["name"])
def test_band_golden(case):
    got = oracle.band_set(case["F"], case["d"], case["q"][0], case["q"][1], case["points"])
    want = np.nonzero(case["expected"])[0]
    np.testing.assert_array_equal(got, want)
    for k, (x, y) in enumerate(case["points"]):
        assert oracle.in_band(oracle.line(case["F"], *case["q"]), case["d"], x, y) == bool(case["expected"][k])


def _exact_member(F, d, xq, yq, xp, yp):
    """Eqs. 2-3 in exact rationals: (a x' + b y' + c)^2 <= d^2 (a^2 + b^2), with a = b = 0 -> no band."""
    Fr = [Fraction(float(v)) for v in F]
    x, y = Fraction(float(xq)), Fraction(float(yq))
    a = Fr[0] * x + Fr[1] * y + Fr[2]
    b = Fr[3] * x + Fr[4] * y + Fr[5]
    c = Fr[6] * x + Fr[7] * y + Fr[8]
    if a == 0 and b == 0:
        return False
    s = a * Fraction(float(xp)) + b * Fraction(float(yp)) + c
    dd = Fraction(float(d))
    return s * s <= dd * dd * (a * a + b * b)


@pytest.mark.parametrize("seed", range(4))
def test_band_against_exact_rationals(seed):
    sc = scenes.random_small(100 + seed, 24, 300, d=12.0)
    A, B = sc.images
    F = sc.pairs[0].F
    seen = 0
    for i in range(A.n):
        got = set(oracle.band_set(F, 12.0, A.xy[i, 0], A.xy[i, 1], B.xy).tolist())
        want = {j for j in range(B.n) if _exact_member(F, 12.0, A.xy[i, 0], A.xy[i, 1], B.xy[j, 0], B.xy[j, 1])}
        assert got == want
        seen += len(want)
    assert seen > 0


def test_known_correspondences_two_view(two_view_scene):
    sc = two_view_scene
    A, B = sc.images
    pr = sc.pairs[0]
    mj, nc = oracle.match_pair(A.xy, A.desc, B.xy, B.desc, pr.F, pr.d, pr.p, pr.q)
    where_b = {int(p): j for j, p in enumerate(B.pid) if p >= 0}
    true = [(i, where_b[int(p)]) for i, p in enumerate(A.pid) if p >= 0 and int(p) in where_b]
    recall = np.mean([mj[i] == j for i, j in true])
    accepted = np.nonzero(mj >= 0)[0]
    wrong = sum(1 for i in accepted if A.pid[i] < 0 or B.pid[mj[i]] != A.pid[i])
    assert recall >= 0.99
    assert wrong <= 0.01 * len(accepted)
    # a planted orientation mistake (the transposed F) must destroy recall: the test has teeth
    Ft = pr.F.reshape(3, 3).T.copy().reshape(9)
    mt, _ = oracle.match_pair(A.xy, A.desc, B.xy, B.desc, Ft, pr.d, pr.p, pr.q)
    assert np.mean([mt[i] == j for i, j in true]) < 0.5


def test_noise_free_projections_satisfy_epipolar_constraint(two_view_scene):
    """x_B^T F x_A = 0 for the generator's F (FP32 rounding only): pins the orientation l_B = F x_A."""
    sc = two_view_scene
    X = sc.info["points"]
    ua, _ = scenes.project(sc.cameras[0], X)
    ub, _ = scenes.project(sc.cameras[1], X)
    for k in range(0, X.shape[0], 50):
        l = oracle.line(sc.pairs[0].F, np.float32(ua[k, 0]), np.float32(ua[k, 1]))
        r = abs(l[0] * ub[k, 0] + l[1] * ub[k, 1] + l[2]) / np.hypot(l[0], l[1])
        assert r < 1e-3


def test_known_correspondences_facade_sample(facade_scene):
    sc = facade_scene
    pairs = sc.pairs[::150]
    outs, ncs = oracle.match_batch(sc.images, pairs)
    for pr, mj in zip(pairs, outs):
        A, B = sc.images[pr.a], sc.images[pr.b]
        where_b = {int(p): j for j, p in enumerate(B.pid) if p >= 0}
        true = [(i, where_b[int(p)]) for i, p in enumerate(A.pid) if p >= 0 and int(p) in where_b]
        assert len(true) >= 50
        assert np.mean([mj[i] == j for i, j in true]) >= 0.99


def test_candidate_fraction_plausible(facade_scene):
    """Sec. 6.2.2 reports |C'| : |F_c| of about 1 : 200 on real data; the synthetic scenes are of that order."""
    sc = facade_scene
    pairs = sc.pairs[:4]
    _, ncs = oracle.match_batch(sc.images, pairs)
    frac = [nc / (sc.images[p.a].n * sc.images[p.b].n) for p, nc in zip(pairs, ncs)]
    assert all(1e-3 < f < 5e-2 for f in frac)


def test_transpose_symmetry_rectified():
    """For F = [[0,0,u],[0,0,v],[-u,-v,0]] (a rotated rectified pair) both directions measure the same
    distance, so membership(A->B, F) is the transpose of membership(B->A, F^T)."""
    rng = np.random.default_rng(3)
    u, v = np.float32(0.6), np.float32(0.8)
    F = np.array([0, 0, u, 0, 0, v, -u, -v, 0], np.float32)
    Ft = F.reshape(3, 3).T.copy().reshape(9)
    xyA = (rng.integers(0, 1280, (60, 2)) / 4.0).astype(np.float32)
    xyB = (rng.integers(0, 1280, (70, 2)) / 4.0).astype(np.float32)
    MAB = np.zeros((60, 70), bool)
    MBA = np.zeros((70, 60), bool)
    for i in range(60):
        MAB[i, oracle.band_set(F, 20.0, xyA[i, 0], xyA[i, 1], xyB)] = True
    for j in range(70):
        MBA[j, oracle.band_set(Ft, 20.0, xyB[j, 0], xyB[j, 1], xyA)] = True
    assert MAB.any()
    np.testing.assert_array_equal(MAB, MBA.T)


def test_repetitive_structure_denser_matches():
    """Sec. 6.2.3 / Fig. 5: with five near-identical copies of a pattern stacked vertically in B, exhaustive
    matching fails the ratio test while the band of a rectified pair isolates the right copy."""
    rng = np.random.default_rng(11)
    base = rng.integers(0, 256, 128).astype(np.int64)
    qd = np.clip(base + rng.normal(0, 4, 128).round(), 0, 255).astype(np.uint8)[None]
    ys = [100.0, 300.0, 500.0, 700.0, 900.0]
    bxy = [[400.0 + 10 * k, y] for k, y in enumerate(ys)]
    bd = [np.clip(base + rng.normal(0, 4, 128).round(), 0, 255) for _ in ys]
    for k in range(6):     # unrelated features on the same row as the query
        bxy.append([50.0 + 100 * k, 101.0])
        bd.append(rng.integers(0, 256, 128))
    bxy = np.array(bxy, np.float32)
    bd = np.array(bd).astype(np.uint8)
    qxy = np.array([[380.0, 100.0]], np.float32)
    guided, _ = oracle.match_pair(qxy, qd, bxy, bd, scenes.RECTIFIED_F, 4.0, 4, 5)
    exhaustive, _ = oracle.match_pair(qxy, qd, bxy, bd, scenes.RECTIFIED_F, np.inf, 4, 5)
    assert guided[0] == 0
    assert exhaustive[0] == -1


def test_stored_two_view_matches(two_view_scene):
    """The stored match list (written by tests/golden/make_golden.py) still comes out of the oracle."""
    path = golden.HERE + "/two_view_matches.txt"
    rows, nc_stored = [], None
    with open(path) as fh:
        for line in fh:
            if line.startswith("# n_cand"):
                nc_stored = int(line.split()[2])
            elif not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    A, B = two_view_scene.images
    pr = two_view_scene.pairs[0]
    mj, nc = oracle.match_pair(A.xy, A.desc, B.xy, B.desc, pr.F, pr.d, pr.p, pr.q)
    assert nc == nc_stored
    np.testing.assert_array_equal(oracle.matches_from_match_j(mj), np.array(rows, np.int32).reshape(-1, 2))
