"""gm_merge_tracks (connected components of the matches) against the oracle, through the C ABI: identical labels."""
import numpy as np
import pytest

from oracle import tracks as ot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06235_gb300 import geomatch
    geomatch.load_library()
    return geomatch


@pytest.mark.parametrize("n,m", [(1, 0), (7, 3), (500, 200), (5000, 9000), (200000, 150000), (100000, 400000)])
def test_random_graphs(gm, n, m):
    rng = np.random.default_rng(n + m)
    edges = rng.integers(0, n, (m, 2)).astype(np.int64)
    with gm.Context(device=0) as ctx:
        lab, nt = ctx.merge_tracks(n, edges)
    want = ot.labels(n, edges)
    np.testing.assert_array_equal(lab, want)
    assert nt == ot.n_tracks(want)


def test_long_chain_and_star(gm):
    n = 300000
    rng = np.random.default_rng(1)
    perm = rng.permutation(n)
    chain = np.stack([perm[:-1], perm[1:]], 1)[rng.permutation(n - 1)]   # one path through every node, shuffled
    star = np.stack([np.full(n - 1, n - 1), np.arange(n - 1)], 1)
    with gm.Context(device=0) as ctx:
        for edges in (chain, star):
            lab, nt = ctx.merge_tracks(n, edges.astype(np.int64))
            assert (lab == 0).all() and nt == 1


def test_facade_match_graph(gm, facade_scene):
    """Tracks of the facade batch's matches: device edges and labels, equal to the oracle."""
    import torch
    sc = facade_scene
    base = np.concatenate([[0], np.cumsum([im.n for im in sc.images])]).astype(np.int64)
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m = ctx.match_pairs(sc.pairs)
        edges = ot.edges_from_matches(base, sc.pairs, off, m)
        lab = torch.empty(int(base[-1]), dtype=torch.int64, device="cuda:0")
        nt = gm.gm_merge_tracks(ctx.h, int(base[-1]), torch.from_numpy(edges).cuda(), lab)
    want = ot.labels(int(base[-1]), edges)
    np.testing.assert_array_equal(lab.cpu().numpy(), want)
    assert nt == ot.n_tracks(want)


def test_bad_endpoint(gm):
    with gm.Context(device=0) as ctx:
        with pytest.raises(gm.GeomatchError) as e:
            ctx.merge_tracks(5, np.array([[0, 5]], np.int64))
        assert e.value.status == gm.GM_ERR_INVALID
