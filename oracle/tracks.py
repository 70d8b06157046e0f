"""Track merging (arXiv 1512.06235, Sec. 6.2 end: tracks are the connected components of the feature matches) --
plain CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests and the CPU-baseline leg of ``bench.py`` may import this module; the product
path never does.  It shares no code with the CUDA library.

Nodes are features (a global index per (image, feature)); every match is an undirected edge.  A track is a
connected component.  The paper finds them with a sequential depth-first search; the result does not depend on the
method, so it is written here as the component labelling of scipy's csgraph.  Reading: each node's label is the
smallest node index in its component (isolated nodes label themselves); the number of tracks counts the
components with at least two nodes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components


def labels(n_nodes: int, edges) -> np.ndarray:
    """int64 [n_nodes]: the smallest node index of each node's component."""
    edges = np.asarray(edges, np.int64).reshape(-1, 2)
    if edges.size and (edges.min() < 0 or edges.max() >= n_nodes):
        raise ValueError("edge endpoint out of range")
    g = sp.coo_matrix((np.ones(len(edges), np.int8), (edges[:, 0], edges[:, 1])), shape=(n_nodes, n_nodes))
    _, comp = connected_components(g, directed=False)
    first = np.full(comp.max() + 1 if n_nodes else 0, n_nodes, np.int64)
    np.minimum.at(first, comp, np.arange(n_nodes, dtype=np.int64))
    return first[comp]


def n_tracks(lab: np.ndarray) -> int:
    """Components with at least two nodes."""
    if lab.size == 0:
        return 0
    roots, counts = np.unique(lab, return_counts=True)
    return int((counts >= 2).sum())


def edges_from_matches(node_base, pairs, pair_off, matches) -> np.ndarray:
    """Edges (global node ids) of the match lists of a batch: pair k = (a, b) with rows (i, j) gives
    (node_base[a] + i, node_base[b] + j)."""
    pair_off = np.asarray(pair_off, np.int64)
    matches = np.asarray(matches, np.int64).reshape(-1, 2)
    k = np.repeat(np.arange(len(pairs)), np.diff(pair_off))
    a = np.array([p.a for p in pairs], np.int64)[k]
    b = np.array([p.b for p in pairs], np.int64)[k]
    base = np.asarray(node_base, np.int64)
    return np.stack([base[a] + matches[:, 0], base[b] + matches[:, 1]], 1)
