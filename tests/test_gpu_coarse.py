"""Coarse stage (Sec. 4) through the C ABI against the oracle: the scale selections and the two-batch match lists
must be identical (integer results), including the preemptive decision of every pair."""
from types import SimpleNamespace

import numpy as np
import pytest

import scenes
from oracle import coarse as oc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06235_gb300 import geomatch
    geomatch.load_library()
    return geomatch


@pytest.fixture(scope="module")
def small_facade():
    return scenes.facade(n_images=10, n_kp=4000, n_points=12000, n_pairs=20, min_covis=20)


def _all_pairs(n, p=4, q=5):
    return [SimpleNamespace(a=a, b=b, p=p, q=q) for a in range(n) for b in range(n) if a != b]


def _check(gm, ctx, images, pairs, eta=20, first=10, min_features=1000, min_matches=4):
    opts = gm.coarse_opts(eta, first, min_features, min_matches)
    off, m, sec = ctx.match_coarse(pairs, opts)
    want = oc.match_coarse(images, pairs, eta, first, min_features, min_matches)
    for k, (rows, ran) in enumerate(want):
        got = m[off[k]:off[k + 1]]
        np.testing.assert_array_equal(got, rows, err_msg=f"pair {k}")
        assert bool(sec[k]) == ran, k
    return off, sec


@pytest.mark.parametrize("eta,first,min_features", [(20, 10, 1000), (30, 15, 1000), (100, 50, 1000), (20, 20, 0),
                                                    (20, 10, 4001), (7, 3, 0)])
def test_selection_matches_oracle(gm, small_facade, eta, first, min_features):
    sc = small_facade
    opts = gm.coarse_opts(eta, first, min_features, 4)
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        for k, im in enumerate(sc.images):
            got = ctx.coarse_selection(k, opts)
            want = oc.select_by_scale(im.scale, eta, first, min_features)
            for g, w in zip(got, want):
                np.testing.assert_array_equal(g, w)


def test_selection_ties_and_signed_zero(gm):
    """Equal scales (lower index first), -0 equal to +0, negative and infinite scales."""
    rng = np.random.default_rng(4)
    n = 3000
    vals = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 2.5, 1e-40, -1e-40], np.float32)
    scale = rng.choice(vals, n).astype(np.float32)
    xy = rng.uniform(0, 100, (n, 2)).astype(np.float32)
    desc = rng.integers(0, 256, (n, 128), dtype=np.uint8)
    with gm.Context(device=0) as ctx:
        ctx.put_image(0, width=100, height=100, xy=xy, scale=scale, desc=desc)
        for eta, first in [(20, 10), (50, 1), (100, 100)]:
            got = ctx.coarse_selection(0, gm.coarse_opts(eta, first, 1000, 4))
            for g, w in zip(got, oc.select_by_scale(scale, eta, first, 1000)):
                np.testing.assert_array_equal(g, w)


def test_match_all_pairs_small_facade(gm, small_facade):
    sc = small_facade
    pairs = _all_pairs(len(sc.images))
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, sec = _check(gm, ctx, sc.images, pairs)
        assert off[-1] > 0
        # a threshold at the median first-batch count: both outcomes of the preemptive rule occur
        c1 = [len(r) for r, _ in oc.match_coarse(sc.images, pairs, min_matches=10 ** 9)]
        thr = int(np.median(c1))
        off, sec = _check(gm, ctx, sc.images, pairs, min_matches=thr)
        assert 0 < sec.sum() < len(pairs)
        # other fractions: the views are rebuilt for the new options
        _check(gm, ctx, sc.images, pairs[:30], eta=30, first=10, min_matches=thr)
        # the fine matcher still works next to the coarse views
        o2, m2 = ctx.match_pairs(sc.pairs[:5])
        assert o2[-1] > 0


@pytest.mark.parametrize("n_first,second", [(4, False), (5, True), (0, False), (60, True)])
def test_preemptive_rule_planted(gm, n_first, second):
    rng = np.random.default_rng(1)
    n = 1000
    sa, sb = rng.permutation(n).astype(np.float32), rng.permutation(n).astype(np.float32)
    da = rng.integers(0, 256, (n, 128), dtype=np.uint8)
    db = rng.integers(0, 256, (n, 128), dtype=np.uint8)
    q1, q2, _ = oc.select_by_scale(sa)
    t = oc.select_by_scale(sb)[2]
    src = np.concatenate([q1[:n_first], q2[:9]])
    dst = t[rng.permutation(t.size)[:src.size]]
    db[dst] = da[src]
    xy = np.stack([np.arange(n) % 40, np.arange(n) // 40], 1).astype(np.float32) + 0.5
    A = SimpleNamespace(width=40, height=25, xy=xy, scale=sa, desc=da)
    B = SimpleNamespace(width=40, height=25, xy=xy, scale=sb, desc=db)
    with gm.Context(device=0) as ctx:
        ctx.put_images({0: A, 1: B})
        off, sec = _check(gm, ctx, [A, B], [SimpleNamespace(a=0, b=1, p=4, q=5)])
        assert bool(sec[0]) is second
        assert off[1] == n_first + (9 if second else 0)


def test_small_images_use_every_feature(gm):
    """Images below min_features: all features in one batch, no second batch; mixed with a large image."""
    sc = scenes.facade(n_images=4, n_kp=np.array([600, 2500, 900, 3000]), n_points=5000, n_pairs=4, min_covis=10)
    pairs = _all_pairs(4)
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, sec = _check(gm, ctx, sc.images, pairs)
        for k, pr in enumerate(pairs):
            if sc.images[pr.a].n < 1000:
                assert sec[k] == 0


def test_device_outputs_cap_and_refresh(gm, small_facade):
    import torch
    sc = small_facade
    pairs = _all_pairs(4)
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images[:4])})
        off_h, m_h, sec_h = ctx.match_coarse(pairs)
        total = int(off_h[-1])
        off = torch.empty(len(pairs) + 1, dtype=torch.int64, device="cuda:0")
        m = torch.empty((total, 2), dtype=torch.int32, device="cuda:0")
        sec = torch.empty(len(pairs), dtype=torch.int32, device="cuda:0")
        n = gm.gm_match_coarse(ctx.h, pairs, off, m, total, sec)
        assert n == total
        np.testing.assert_array_equal(off.cpu().numpy(), off_h)
        np.testing.assert_array_equal(m.cpu().numpy(), m_h)
        np.testing.assert_array_equal(sec.cpu().numpy(), sec_h)
        small = np.full((total - 1, 2), -7, np.int32)
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_match_coarse(ctx.h, pairs, np.empty(len(pairs) + 1, np.int64), small, total - 1)
        assert e.value.status == gm.GM_ERR_NOMEM and e.value.required == total and (small == -7).all()
        # selection lists of mixed kinds (device q1, host q2 and t) are refused, nothing written
        q1 = torch.full((8000,), -5, dtype=torch.int32, device="cuda:0")
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_coarse_selection(ctx.h, 0, q1, np.empty(8000, np.int32), np.empty(8000, np.int32), 8000)
        assert e.value.status == gm.GM_ERR_INVALID and bool((q1 == -5).all())
        # putting an image again with other scales refreshes its views
        im = sc.images[0]
        rev = SimpleNamespace(width=im.width, height=im.height, xy=im.xy, desc=im.desc, scale=im.scale[::-1].copy())
        ctx.put_image(0, rev)
        imgs = [rev] + list(sc.images[1:4])
        _check(gm, ctx, imgs, pairs)
        # evicting an image drops its views; matching it is then NOT_FOUND
        ctx.evict(1)
        with pytest.raises(gm.GeomatchError) as e:
            ctx.match_coarse(pairs[:3])
        assert e.value.status == gm.GM_ERR_NOT_FOUND


def test_full_facade_all_pairs_sampled(gm, facade_scene):
    """The benchmark's launch: every unordered pair of the 100 facade images (4950) in one call; 40 sampled pairs
    against the oracle, rows and second-batch flags."""
    sc = facade_scene
    n = len(sc.images)
    pairs = [SimpleNamespace(a=a, b=b, p=4, q=5) for a in range(n) for b in range(a + 1, n)]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m, sec = ctx.match_coarse(pairs)
    pick = np.random.default_rng(9).choice(len(pairs), 40, replace=False)
    want = oc.match_coarse(sc.images, [pairs[k] for k in pick])
    for k, (rows, ran) in zip(pick, want):
        np.testing.assert_array_equal(m[off[k]:off[k + 1]], rows, err_msg=f"pair {k}")
        assert bool(sec[k]) == ran


def test_errors(gm):
    rng = np.random.default_rng(2)
    n = 1200
    xy = rng.uniform(0, 50, (n, 2)).astype(np.float32)
    desc = rng.integers(0, 256, (n, 128), dtype=np.uint8)
    scale = rng.random(n).astype(np.float32)
    nan_scale = scale.copy()
    nan_scale[17] = np.nan
    with gm.Context(device=0) as ctx:
        ctx.put_image(0, width=50, height=50, xy=xy, scale=scale, desc=desc)
        ctx.put_image(1, width=50, height=50, xy=xy, scale=None, desc=desc)
        ctx.put_image(2, width=50, height=50, xy=xy, scale=nan_scale, desc=desc)
        pr = lambda a, b: SimpleNamespace(a=a, b=b, p=4, q=5)
        for pairs, opts, status in [
            ([pr(0, 1)], None, gm.GM_ERR_INVALID),                          # no scales
            ([pr(0, 2)], None, gm.GM_ERR_INVALID),                          # a NaN scale
            ([pr(0, 9)], None, gm.GM_ERR_NOT_FOUND),
            ([pr(0, 0)], gm.coarse_opts(20, 30, 1000, 4), gm.GM_ERR_INVALID),   # first > eta
            ([pr(0, 0)], gm.coarse_opts(0, 0, 1000, 4), gm.GM_ERR_INVALID),
            ([SimpleNamespace(a=0, b=0, p=5, q=5)], None, gm.GM_ERR_INVALID),
        ]:
            with pytest.raises(gm.GeomatchError) as e:
                ctx.match_coarse(pairs, opts)
            assert e.value.status == status
        ctx.match_coarse([pr(0, 0)])   # builds internal views
        # internal images are not addressable through the public calls
        with pytest.raises(gm.GeomatchError) as e:
            ctx.match_pairs([gm.make_pair(-1, 0, np.eye(3), 4.0)])
        assert e.value.status == gm.GM_ERR_NOT_FOUND
        with pytest.raises(gm.GeomatchError) as e:
            ctx.evict(-1)
        assert e.value.status == gm.GM_ERR_NOT_FOUND
