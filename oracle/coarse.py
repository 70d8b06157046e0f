"""Coarse-stage matching (arXiv 1512.06235, Sec. 4): high-scale feature selection and the hybrid preemptive
schedule -- plain CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests and the CPU-baseline leg of ``bench.py`` may import this module; the product
path never does.  It shares no code with the CUDA library; the matching itself is the plain FP64 C oracle of
Sec. 6.2 (``oracle.match_pair``) run with an unbounded band, i.e. exhaustive nearest / second-nearest search.

Selection (Sec. 4): every image keeps its eta % features of the largest scale.  Readings: the count is
floor(n * eta / 100); equal scales are ordered by the lower feature index first; an image with fewer than
``min_features`` features (the paper's 1000) keeps all of them.

Preemptive schedule (Sec. 4): for a pair (A, B) the first ``first`` % of A's features by scale are the queries of a
first batch against B's selected features; the rest of A's selection (ranks first % .. eta %) is matched against
the same targets only when the first batch gave more than ``min_matches`` (the paper's 4) matches.  Readings: an
image below ``min_features`` is matched with all of its features in the first batch and has no second batch; the
optional early termination once "enough" matches exist is not applied; the match list of a pair is the first
batch's rows followed by the second batch's rows, each sorted by the query's feature index.
"""
from __future__ import annotations

import numpy as np

import oracle


def select_by_scale(scale, eta: int = 20, first: int = 10, min_features: int = 1000):
    """(q1, q2, t): ascending feature indices of the first query batch, the second query batch and the targets."""
    scale = np.asarray(scale, np.float32)
    n = scale.shape[0]
    if n < min_features:
        every = np.arange(n, dtype=np.int32)
        return every, np.zeros(0, np.int32), every
    rank = sorted(range(n), key=lambda i: (-float(scale[i]), i))   # descending scale, then lower index
    k_t = n * eta // 100
    k_1 = n * first // 100
    t = np.sort(np.array(rank[:k_t], np.int32))
    q1 = np.sort(np.array(rank[:k_1], np.int32))
    q2 = np.sort(np.array(rank[k_1:k_t], np.int32))
    return q1, q2, t


def _batch(img_a, img_b, qa, tb, p, q):
    """Rows (feature of A, feature of B) of the queries qa of A against the targets tb of B, unbounded band."""
    if qa.size == 0 or tb.size == 0:
        return np.zeros((0, 2), np.int32)
    F = np.eye(3, dtype=np.float32).reshape(9)   # unused: the band is unbounded
    mj, _ = oracle.match_pair(img_a.xy[qa], img_a.desc[qa], img_b.xy[tb], img_b.desc[tb], F, float("inf"), p, q)
    i = np.nonzero(mj >= 0)[0]
    return np.stack([qa[i], tb[mj[i]]], 1).astype(np.int32).reshape(-1, 2)


def match_coarse(images, pairs, eta: int = 20, first: int = 10, min_features: int = 1000, min_matches: int = 4):
    """Per pair (objects with a, b, p, q): (rows int32 [m, 2], second batch run?)."""
    sel = {}
    for k in {pr.a for pr in pairs} | {pr.b for pr in pairs}:
        sel[k] = select_by_scale(images[k].scale, eta, first, min_features)
    out = []
    for pr in pairs:
        q1, q2, _ = sel[pr.a]
        t = sel[pr.b][2]
        r1 = _batch(images[pr.a], images[pr.b], q1, t, pr.p, pr.q)
        second = r1.shape[0] > min_matches and q2.size > 0
        r2 = _batch(images[pr.a], images[pr.b], q2, t, pr.p, pr.q) if second else np.zeros((0, 2), np.int32)
        out.append((np.concatenate([r1, r2]), second))
    return out
