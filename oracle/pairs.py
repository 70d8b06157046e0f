"""Candidate image pairs from point-camera co-visibility (arXiv 1512.06235, Sec. 6.1) -- plain CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests and the CPU-baseline leg of ``bench.py`` may import this module; the product
path never does.  It shares no code with the CUDA library.

What it computes.  Each 3D point of the coarse model is seen by a set of cameras.  For two images,
P_cv(I_i, I_j) = Points(C_i) intersected with Points(C_j) is the set of points both see.  The candidate images of
a query image q are S_q = { i != q : |P_cv(q, i)| > T }, of which only the top k ranked by |P_cv| are kept; the pairs
to match are the unique unordered pairs {q, i} over all queries.  Reading where the paper is silent: ties in the
ranking go to the lower image index; a pair appears once however many of its two images selected it; rows are
(a, b, count) with a < b, sorted by (a, b).

The co-visible counts are the entries of C = M M^T for the camera-by-point incidence matrix M (M[c, p] = 1 iff
camera c sees point p): C[i, j] counts the points in both sets.  The product is scipy's sparse matmul; the ranking
and the union are plain loops.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def incidence(n_cams: int, point_off, point_cams) -> sp.csr_matrix:
    """Camera-by-point incidence M (0/1).  Every point lists distinct cameras in [0, n_cams)."""
    point_off = np.asarray(point_off, np.int64)
    point_cams = np.asarray(point_cams, np.int64)
    n_points = point_off.size - 1
    if point_cams.size and (point_cams.min() < 0 or point_cams.max() >= n_cams):
        raise ValueError("camera index out of range")
    pts = np.repeat(np.arange(n_points, dtype=np.int64), np.diff(point_off))
    M = sp.csr_matrix((np.ones(point_cams.size, np.int64), (point_cams, pts)), shape=(n_cams, n_points))
    if M.nnz != point_cams.size or (M.data != 1).any():
        raise ValueError("a point lists the same camera twice")
    return M


def covisibility(n_cams: int, point_off, point_cams) -> np.ndarray:
    """Dense co-visible counts C[i, j] = |Points(C_i) & Points(C_j)| (int64, diagonal = |Points(C_i)|)."""
    M = incidence(n_cams, point_off, point_cams)
    return np.asarray((M @ M.T).todense(), dtype=np.int64)


def select_pairs(n_cams: int, point_off, point_cams, threshold: int, top_k: int) -> np.ndarray:
    """Rows (a, b, count), a < b, sorted: the union over queries q of {q, i} for the top_k images i of S_q."""
    C = covisibility(n_cams, point_off, point_cams)
    chosen = set()
    for q in range(n_cams):
        i = np.nonzero((C[q] > threshold) & (np.arange(n_cams) != q))[0]   # S_q
        i = i[np.lexsort((i, -C[q, i]))][:max(top_k, 0)]                    # by count, descending; ties: lower index
        chosen.update((min(q, int(t)), max(q, int(t))) for t in i)
    rows = sorted(chosen)
    out = np.zeros((len(rows), 3), np.int64)
    for r, (a, b) in enumerate(rows):
        out[r] = (a, b, C[a, b])
    return out
