"""Pins of the track-merging oracle: breadth-first search on small graphs, closed forms (CPU)."""
from collections import deque

import numpy as np
import pytest

from oracle import tracks as ot


def _bfs_labels(n, edges):
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    lab = [-1] * n
    for s in range(n):   # visiting sources in increasing order labels each component with its smallest node
        if lab[s] >= 0:
            continue
        lab[s] = s
        dq = deque([s])
        while dq:
            x = dq.popleft()
            for y in adj[x]:
                if lab[y] < 0:
                    lab[y] = s
                    dq.append(y)
    return np.array(lab, np.int64)


@pytest.mark.parametrize("seed", range(8))
def test_labels_match_bfs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    m = int(rng.integers(0, 2 * n))
    edges = rng.integers(0, n, (m, 2))
    np.testing.assert_array_equal(ot.labels(n, edges), _bfs_labels(n, edges.tolist()))


def test_closed_forms():
    n = 10
    chain = np.stack([np.arange(n - 1), np.arange(1, n)], 1)[::-1]
    assert (ot.labels(n, chain) == 0).all() and ot.n_tracks(ot.labels(n, chain)) == 1
    star = np.stack([np.full(n - 1, 7), np.r_[0:7, 8:10]], 1)
    assert (ot.labels(n, star) == 0).all()
    lab = ot.labels(n, np.zeros((0, 2), np.int64))
    np.testing.assert_array_equal(lab, np.arange(n)) and ot.n_tracks(lab) == 0
    two = np.array([[9, 4], [4, 6], [1, 3], [3, 3]])   # a self loop adds nothing
    np.testing.assert_array_equal(ot.labels(n, two), [0, 1, 2, 1, 4, 5, 4, 7, 8, 4])
    assert ot.n_tracks(ot.labels(n, two)) == 2


def test_edges_from_matches():
    class P:
        def __init__(self, a, b):
            self.a, self.b = a, b
    e = ot.edges_from_matches([0, 5, 9], [P(0, 2), P(1, 0)], [0, 2, 3], [[0, 1], [4, 3], [2, 2]])
    np.testing.assert_array_equal(e, [[0, 10], [4, 12], [7, 2]])
