"""The resident-image cache under a memory budget (GM_OPT_EVICT_LRU): least recently used images are evicted to make
room for a put, never one of the images being put; without the option the put is refused and nothing changes.
Matches over the images that stay resident equal those of an unlimited context."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06235_gb300 import geomatch
    geomatch.load_library()
    return geomatch


@pytest.fixture(scope="module")
def small_scene():
    return scenes.facade(n_images=8, n_kp=2000, n_points=6000, n_pairs=12, min_covis=10)


def _pair(gm, sc, a, b):
    F = next((p.F for p in sc.pairs if (p.a, p.b) == (a, b)), None)
    return gm.make_pair(a, b, F if F is not None else scenes.fundamental(sc.cameras[a], sc.cameras[b]), 4.0)


def test_lru_eviction(gm, small_scene):
    sc = small_scene
    with gm.Context(device=0) as ref:   # bytes per image (same size and keypoint count) and reference matches
        ref.put_images({k: im for k, im in enumerate(sc.images)})
        per_image = gm.gm_image_cache_stats(ref.h)["bytes"] // len(sc.images)
        want = {ab: ref.match_pairs([_pair(gm, sc, *ab)])[1] for ab in [(0, 4), (1, 5)]}
    def fits(budget):   # four images, the work buffers of a small match, and a re-put into the same blocks
        with gm.Context(device=0, mem_budget_bytes=budget) as ctx:
            try:
                ctx.put_images({k: sc.images[k] for k in range(4)})
                ctx.match_pairs([_pair(gm, sc, 0, 1)])
                ctx.put_images({k: sc.images[k] for k in range(4)})
                return True
            except gm.GeomatchError as e:
                assert e.status == gm.GM_ERR_BUDGET
                return False

    lo, hi = per_image * 4, per_image * 4 + (1 << 30)   # the smallest budget that fits, to a quarter image
    assert fits(hi)
    while hi - lo > per_image // 4:
        mid = (lo + hi) // 2
        if fits(mid):
            hi = mid
        else:
            lo = mid
    budget = hi
    with gm.Context(device=0, mem_budget_bytes=budget) as ctx:
        ctx.put_images({k: sc.images[k] for k in range(4)})        # images 0..3, put in this order
        ctx.match_pairs([_pair(gm, sc, 0, 1)])                      # 0 and 1 are now the most recently used
        # without eviction the fifth image does not fit: refused, nothing changes
        with pytest.raises(gm.GeomatchError) as e:
            ctx.put_images({4: sc.images[4], 5: sc.images[5]})
        assert e.value.status == gm.GM_ERR_BUDGET
        assert all(gm.gm_image_info(ctx.h, k) == sc.images[k].n for k in range(4))
        ctx.set_option(gm.GM_OPT_EVICT_LRU, 1)
        gm.gm_image_pin(ctx.h, 2, True)                             # the least recently used, but pinned
        ctx.put_images({4: sc.images[4], 5: sc.images[5]})
        resident = [k for k in range(6) if gm.gm_image_info(ctx.h, k) is not None]
        assert 4 in resident and 5 in resident and 2 in resident
        assert 3 not in resident                                    # the least recently used unpinned image went first
        assert len(resident) == 4
        gm.gm_image_pin(ctx.h, 2, False)
        with pytest.raises(gm.GeomatchError) as e:                  # pins count: one pin, one unpin
            gm.gm_image_pin(ctx.h, 2, False)
        assert e.value.status == gm.GM_ERR_INVALID
        stats = gm.gm_image_cache_stats(ctx.h)
        assert stats["evicted"] >= 1 and stats["bytes"] <= budget
        for ab in [(0, 4), (1, 5)]:
            if {*ab} <= set(resident):
                np.testing.assert_array_equal(ctx.match_pairs([_pair(gm, sc, *ab)])[1], want[ab])
        with pytest.raises(gm.GeomatchError) as e:                  # an evicted image is gone
            ctx.match_pairs([_pair(gm, sc, 3, 4)])
        assert e.value.status == gm.GM_ERR_NOT_FOUND
        # a put that could not fit even after evicting every other image is refused
        big = {10 + k: sc.images[k % 8] for k in range(40)}
        with pytest.raises(gm.GeomatchError) as e:
            ctx.put_images(big)
        assert e.value.status == gm.GM_ERR_BUDGET
        assert gm.gm_image_info(ctx.h, 4) == sc.images[4].n          # and nothing was evicted for it
        assert [k for k in range(6) if gm.gm_image_info(ctx.h, k) is not None] == resident
