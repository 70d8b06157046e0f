"""Pins of the coarse-stage oracle (Sec. 4): scale selection by closed forms, the preemptive rule on planted
matches, and the batch rows against a pure-Python brute force (CPU)."""
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import coarse as oc


def _img(scale, desc, xy=None):
    n = len(scale)
    if xy is None:
        xy = np.stack([np.arange(n) % 64, np.arange(n) // 64], 1).astype(np.float32) + 0.5
    return SimpleNamespace(scale=np.asarray(scale, np.float32), desc=np.asarray(desc, np.uint8), xy=xy, n=n)


def test_selection_closed_forms():
    rng = np.random.default_rng(0)
    n = 1234
    perm = rng.permutation(n)                      # scale of feature i = perm[i]: the top k are perm >= n - k
    q1, q2, t = oc.select_by_scale(perm.astype(np.float32), 20, 10, 1000)
    k_t, k_1 = n * 20 // 100, n * 10 // 100        # 246 and 123
    assert t.tolist() == np.nonzero(perm >= n - k_t)[0].tolist()
    assert q1.tolist() == np.nonzero(perm >= n - k_1)[0].tolist()
    assert q2.tolist() == np.nonzero((perm >= n - k_t) & (perm < n - k_1))[0].tolist()
    # equal scales: the lower indices first
    q1, q2, t = oc.select_by_scale(np.ones(1001, np.float32), 20, 10, 1000)
    assert t.tolist() == list(range(200)) and q1.tolist() == list(range(100)) and q2.tolist() == list(range(100, 200))
    # below min_features: everything, one batch
    q1, q2, t = oc.select_by_scale(rng.random(999), 20, 10, 1000)
    assert q1.tolist() == list(range(999)) and t.tolist() == list(range(999)) and q2.size == 0


def _planted(n_first, n_second, seed=1):
    """A and B of 1000 features; B's selected features hold exact copies of `n_first` of A's first-batch queries
    and `n_second` of its second-batch queries; every other descriptor is uniform noise."""
    rng = np.random.default_rng(seed)
    n = 1000
    sa, sb = rng.permutation(n).astype(np.float32), rng.permutation(n).astype(np.float32)
    da = rng.integers(0, 256, (n, 128), dtype=np.uint8)
    db = rng.integers(0, 256, (n, 128), dtype=np.uint8)
    q1, q2, _ = oc.select_by_scale(sa)
    t = oc.select_by_scale(sb)[2]
    src = np.concatenate([q1[:n_first], q2[:n_second]])
    dst = t[rng.permutation(t.size)[:src.size]]
    db[dst] = da[src]
    want = dict(zip(src.tolist(), dst.tolist()))
    return _img(sa, da), _img(sb, db), q1, q2, want


@pytest.mark.parametrize("n_first,second", [(4, False), (5, True), (0, False), (30, True)])
def test_preemptive_rule(n_first, second):
    A, B, q1, q2, want = _planted(n_first, 7)
    (rows, ran), = oc.match_coarse([A, B], [SimpleNamespace(a=0, b=1, p=4, q=5)])
    assert ran is second
    first_rows = [(i, j) for i, j in want.items() if i in set(q1.tolist())]
    second_rows = [(i, j) for i, j in want.items() if i in set(q2.tolist())]
    expect = sorted(first_rows) + (sorted(second_rows) if second else [])
    assert [tuple(r) for r in rows.tolist()] == expect


def _brute(da, db, qa, tb, p, q):
    rows = []
    for i in qa:
        d = sorted((int(((da[i].astype(np.int64) - db[j].astype(np.int64)) ** 2).sum()), j) for j in tb)
        if len(d) >= 2 and q * q * d[0][0] < p * p * d[1][0]:   # fewer than two candidates: no ratio, no match
            rows.append((int(i), int(d[0][1])))
    return rows


def test_batches_against_brute_force():
    """Small images with a low min_features: the two batches' rows equal a pure-Python exhaustive search over the
    selected features."""
    rng = np.random.default_rng(3)
    na, nb = 60, 45
    base = rng.integers(0, 256, (80, 128))
    da = np.clip(base[rng.integers(0, 80, na)] + rng.normal(0, 6, (na, 128)), 0, 255).astype(np.uint8)
    db = np.clip(base[rng.integers(0, 80, nb)] + rng.normal(0, 6, (nb, 128)), 0, 255).astype(np.uint8)
    A, B = _img(rng.random(na), da), _img(rng.random(nb), db)
    for eta, first in [(50, 25), (100, 50), (20, 10)]:
        (rows, ran), = oc.match_coarse([A, B], [SimpleNamespace(a=0, b=1, p=4, q=5)], eta, first, 10, 0)
        q1, q2, _ = oc.select_by_scale(A.scale, eta, first, 10)
        t = oc.select_by_scale(B.scale, eta, first, 10)[2]
        r1 = _brute(da, db, q1, t, 4, 5)
        r2 = _brute(da, db, q2, t, 4, 5) if len(r1) > 0 and q2.size else []
        assert ran == (len(r1) > 0 and q2.size > 0)
        assert [tuple(r) for r in rows.tolist()] == r1 + r2
