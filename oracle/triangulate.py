"""Triangulation of feature tracks (arXiv 1512.06235, Sec. 6.3: tracks are triangulated with a standard
least-squares method) -- plain CPU oracle, FP64.

Two track definitions are covered.  ``image_tracks`` follows Sec. 6.3's order: every query image's features form
tracks from that image's matches in all its candidate images, and each such track is triangulated on its own,
image by image (which duplicates points: a feature pair matched in both directions is triangulated once for each
image).  ``triangulate_tracks`` triangulates the merged tracks (the connected components of all matches), the
result after Sec. 6.3's merging step.

TEST INFRASTRUCTURE ONLY: the tests and the CPU-baseline leg of ``bench.py`` may import this module; the product
path never does.  It shares no code with the CUDA library.

Each observation of a track -- camera matrix P (3 x 4) and image point (x, y) -- gives two linear equations in the
homogeneous point X = (X, Y, Z, 1): (x P3 - P1) X = 0 and (y P3 - P2) X = 0, where Pk is row k of P.  The point is
the linear least-squares solution of these equations with the fourth coordinate fixed to 1, i.e. the solution of
the 3 x 3 normal equations (A3^T A3) X = -A3^T a4 for the stacked rows A = [A3 | a4].  Readings: every component
with at least two observations is a track (tracks are ordered by their smallest node); a singular system gives NaN.
"""
from __future__ import annotations

import numpy as np


def triangulate(P_list, xy_list) -> np.ndarray:
    """One track: P_list [n][3, 4], xy_list [n][2] -> X (3,) in FP64."""
    rows = []
    for P, (x, y) in zip(P_list, xy_list):
        P = np.asarray(P, np.float64)
        rows.append(float(x) * P[2] - P[0])
        rows.append(float(y) * P[2] - P[1])
    A = np.array(rows, np.float64)
    M = A[:, :3].T @ A[:, :3]
    b = -(A[:, :3].T @ A[:, 3])
    try:
        return np.linalg.solve(M, b)
    except np.linalg.LinAlgError:
        return np.full(3, np.nan)


def triangulate_tracks(P_per_image, xy_per_image, labels) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Tracks from image-major node labels.  P_per_image [n_images][3, 4]; xy_per_image[k] float [n_k, 2];
    labels int64 [sum n_k].  Returns (roots int64 [T], n_views int32 [T], X float64 [T, 3]) ordered by root."""
    counts = np.array([len(xy) for xy in xy_per_image], np.int64)
    base = np.concatenate([[0], np.cumsum(counts)])
    labels = np.asarray(labels, np.int64)
    order = np.argsort(labels, kind="stable")
    lab_sorted = labels[order]
    roots, start, size = np.unique(lab_sorted, return_index=True, return_counts=True)
    keep = size >= 2
    out_X, out_n = [], []
    for r, s, n in zip(roots[keep], start[keep], size[keep]):
        nodes = order[s:s + n]
        img = np.searchsorted(base, nodes, side="right") - 1
        Ps = [P_per_image[k] for k in img]
        xys = [xy_per_image[k][v - base[k]] for k, v in zip(img, nodes)]
        out_X.append(triangulate(Ps, xys))
        out_n.append(n)
    return roots[keep].astype(np.int64), np.array(out_n, np.int32), np.array(out_X, np.float64).reshape(-1, 3)


def image_tracks(P_per_image, xy_per_image, pairs, pair_matches):
    """Per-image tracks (Sec. 6.3).  For every query image q and feature k: the observation (q, k) itself, then
    (c, j) for every pair (q, c) -- in the order of ``pairs`` -- in which k matched j.  Every track with at least
    two observations is triangulated with ``triangulate``.

    P_per_image [n_images][3, 4]; xy_per_image[k] float [n_k, 2]; pairs: (a, b) image indices, a the query image;
    pair_matches[p]: int [m_p, 2] rows (i, j) of pair p (feature i of a, feature j of b).  Nodes are numbered
    image-major (node = features of the images before + feature index).  Returns (nodes int64 [T] -- the query
    node of each track --, n_views int32 [T], X float64 [T, 3]), tracks in increasing order of their query node."""
    counts = [len(xy) for xy in xy_per_image]
    base = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    obs = {}
    for (a, b), rows in zip(pairs, pair_matches):
        for i, j in np.asarray(rows, np.int64).reshape(-1, 2):
            v = int(base[a] + i)
            if v not in obs:
                obs[v] = [(int(a), int(i))]
            obs[v].append((int(b), int(j)))
    nodes = sorted(obs)
    X = [triangulate([P_per_image[k] for k, _ in obs[v]], [xy_per_image[k][f] for k, f in obs[v]]) for v in nodes]
    return (np.array(nodes, np.int64), np.array([len(obs[v]) for v in nodes], np.int32),
            np.array(X, np.float64).reshape(-1, 3))


def camera_matrix(cam) -> np.ndarray:
    """P = K [R | t] of a pinhole camera (x ~ P X)."""
    return cam.K @ np.hstack([cam.R, cam.t.reshape(3, 1)])
