"""gm_match_pairs_approx (the paper's approximate search: overlapping grids, centre-most cells, dual-line groups)
through the C ABI against the oracle: identical match lists (integer results) and identical group and candidate
counts, since both sides take the geometric decisions in the same FP32 arithmetic."""
from types import SimpleNamespace

import numpy as np
import pytest

import scenes
from oracle import approx as oa

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06235_gb300 import geomatch
    geomatch.load_library()
    return geomatch


def _want(images, pairs, cell_scale):
    rows, groups, cands = [], 0, 0
    for pr in pairs:
        A, B = images[pr.a], images[pr.b]
        mj, g, c = oa.match_pair(A.xy, A.desc, B.xy, B.desc, B.width, B.height, pr.F, pr.d, pr.p, pr.q, cell_scale,
                                 with_stats=True)
        i = np.nonzero(mj >= 0)[0]
        rows.append(np.stack([i, mj[i]], 1).astype(np.int32).reshape(-1, 2))
        groups += g
        cands += c
    return rows, groups, cands


def _check(gm, ctx, images, pairs, cell_scale=1.0):
    off, m, st = ctx.match_pairs_approx([gm.make_pair(p.a, p.b, p.F, p.d, p.p, p.q) for p in pairs], cell_scale)
    rows, groups, cands = _want(images, pairs, cell_scale)
    for k, r in enumerate(rows):
        np.testing.assert_array_equal(m[off[k]:off[k + 1]], r, err_msg=f"pair {k}")
    assert st["n_groups"] == groups and st["n_candidates"] == cands
    return off, m, st


@pytest.mark.parametrize("cell_scale", [1.0, 1.5, 2.0])
def test_two_view(gm, two_view_scene, cell_scale):
    sc = two_view_scene
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m, st = _check(gm, ctx, sc.images, sc.pairs + [scenes.Pair(1, 0, sc.pairs[0].F.reshape(3, 3).T.reshape(9),
                                                                         4.0)], cell_scale)
        assert off[1] > 500 and st["n_groups"] > 50


def test_wide_band_compacts_in_rounds(gm, two_view_scene):
    """A band so wide that C' of most groups exceeds the 512-entry list, so C' is compacted from the bitmap in rounds:
    the same matches and counts as the oracle."""
    sc = two_view_scene
    pr = sc.pairs[0]
    wide = [SimpleNamespace(a=pr.a, b=pr.b, F=pr.F, d=150.0, p=4, q=5)]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m, st = _check(gm, ctx, sc.images, wide, 1.5)
    assert st["n_candidates"] > 512 * sc.images[pr.a].n


def test_facade_full_batch_sampled(gm, facade_scene):
    """The whole 1200-pair facade batch in one call (the benchmark's launch); eight sampled pairs against the
    oracle."""
    sc = facade_scene
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m, st = ctx.match_pairs_approx([gm.make_pair(p.a, p.b, p.F, p.d, p.p, p.q) for p in sc.pairs])
    pick = np.random.default_rng(12).choice(len(sc.pairs), 8, replace=False)
    rows, _, _ = _want(sc.images, [sc.pairs[k] for k in pick], 1.0)
    for k, r in zip(pick, rows):
        np.testing.assert_array_equal(m[off[k]:off[k + 1]], r, err_msg=f"pair {k}")
    assert st["n_groups"] > 100000


def test_facade_pairs(gm, facade_scene):
    sc = facade_scene
    pairs = sc.pairs[:6]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m, st = _check(gm, ctx, sc.images, pairs)
        # the exact path finds a superset of most of these matches: the approximation loses little here
        eo, em = ctx.match_pairs([gm.make_pair(p.a, p.b, p.F, p.d, p.p, p.q) for p in pairs])
        exact = {(k, int(i), int(j)) for k in range(len(pairs)) for i, j in em[eo[k]:eo[k + 1]]}
        approx = {(k, int(i), int(j)) for k in range(len(pairs)) for i, j in m[off[k]:off[k + 1]]}
        assert len(approx & exact) > 0.9 * len(exact)


def test_random_small_and_edges(gm):
    """Ragged sizes and tie-heavy descriptors, a pair whose lines all miss B, F = 0 (no lines), one query row (every
    line the same: one group), n_B = 1 and 0, n_A = 0."""
    rng = np.random.default_rng(7)
    images, pairs = [], []
    for s, d, lv in [(30, 1.0, 256), (31, 3.0, 4), (32, 6.5, 2)]:
        sc = scenes.random_small(s, int(rng.integers(50, 700)), int(rng.integers(50, 700)), d=d, desc_levels=lv)
        a = len(images)
        images += sc.images
        pairs.append(SimpleNamespace(a=a, b=a + 1, F=np.asarray(sc.pairs[0].F, np.float32), d=d, p=4, q=5))
    W, H = images[1].width, images[1].height
    F0 = pairs[0].F
    pairs.append(SimpleNamespace(a=0, b=1, F=np.array([0, 0, 0, 0, 0, -1, 0, 1, 10000], np.float32), d=4.0, p=4, q=5))
    pairs.append(SimpleNamespace(a=0, b=1, F=np.zeros(9, np.float32), d=4.0, p=4, q=5))
    mk = lambda xy, desc: SimpleNamespace(width=W, height=H, xy=np.asarray(xy, np.float32),
                                          scale=np.ones(len(xy), np.float32), desc=np.asarray(desc, np.uint8))
    row = mk(np.stack([rng.uniform(0, W, 300), np.full(300, 17.25)], 1), rng.integers(0, 256, (300, 128)))
    one = mk([[3.5, 4.5]], rng.integers(0, 256, (1, 128)))
    none = mk(np.zeros((0, 2)), np.zeros((0, 128)))
    r, o, z = len(images), len(images) + 1, len(images) + 2
    images += [row, one, none]
    rect = np.array([0, 0, 0, 0, 0, -1, 0, 1, 0], np.float32)
    pairs += [SimpleNamespace(a=r, b=1, F=rect, d=2.0, p=4, q=5), SimpleNamespace(a=0, b=o, F=F0, d=4.0, p=4, q=5),
              SimpleNamespace(a=0, b=z, F=F0, d=4.0, p=4, q=5), SimpleNamespace(a=z, b=0, F=F0, d=4.0, p=4, q=5)]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(images)})
        off, m, st = _check(gm, ctx, images, pairs)
        assert off[4] == off[3] and off[5] == off[4]   # missing lines and F = 0: no matches


def test_device_buffers_cap_and_errors(gm, two_view_scene):
    import torch
    sc = two_view_scene
    gp = [gm.make_pair(p.a, p.b, p.F, p.d, p.p, p.q) for p in sc.pairs]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off_h, m_h, _ = ctx.match_pairs_approx(gp)
        total = int(off_h[-1])
        off = torch.empty(2, dtype=torch.int64, device="cuda:0")
        m = torch.empty((total, 2), dtype=torch.int32, device="cuda:0")
        n, _ = gm.gm_match_pairs_approx(ctx.h, gp, off, m, total)
        assert n == total
        np.testing.assert_array_equal(m.cpu().numpy(), m_h)
        np.testing.assert_array_equal(off.cpu().numpy(), off_h)
        small = np.full((total - 1, 2), -3, np.int32)
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_match_pairs_approx(ctx.h, gp, np.empty(2, np.int64), small, total - 1)
        assert e.value.status == gm.GM_ERR_NOMEM and e.value.required == total and (small == -3).all()
        F = sc.pairs[0].F
        for pair, scale in [(gm.make_pair(0, 1, F, float("inf")), 1.0), (gm.make_pair(0, 1, F, 0.25), 1.0),
                            (gm.make_pair(0, 1, F, 4.0), 0.0), (gm.make_pair(0, 7, F, 4.0), 1.0)]:
            with pytest.raises(gm.GeomatchError) as e:
                gm.gm_match_pairs_approx(ctx.h, [pair], np.empty(2, np.int64), np.empty((4, 2), np.int32), 4, scale)
            assert e.value.status in (gm.GM_ERR_INVALID, gm.GM_ERR_NOT_FOUND)
