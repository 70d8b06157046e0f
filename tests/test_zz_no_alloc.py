"""gm_band_candidates_static (no allocation, fixed device scratch) against gm_band_candidates, through the C ABI.

The entry point serves callers that cannot allocate during the call: a process whose device memory is taken (the
context's budget is used up by resident images), or a loop that must not stall on cudaMalloc / cudaFree.  Two
calls in a row must both reproduce the allocating entry point exactly (the scratch is reused and must be cleared
by every call); a call must leave the device's free memory and the context's work buffers as they were, and it
must work in a context whose budget has no room for the allocating call's workspace.  The file is collected last
so that it also runs after every other GPU test.
"""
import math

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


def _static(gm, ctx, pair, q0, qn, cap):
    import torch
    off = torch.zeros(qn + 1, dtype=torch.int64, device="cuda:0")
    cand = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda:0")
    n = gm.gm_band_candidates_static(ctx.h, pair, q0, qn, off, cand, cap)
    torch.cuda.synchronize()
    return off.cpu().numpy(), cand[:n].cpu().numpy(), n


@pytest.mark.parametrize("d", [0.0, 4.0, 25.0, math.inf])
def test_static_equals_allocating_entry_point(gm, two_view_scene, d):
    sc = two_view_scene
    pr = sc.pairs[0]
    with gm.Context(device=0) as ctx:
        ctx.put_image(0, sc.images[pr.a])
        ctx.put_image(1, sc.images[pr.b])
        pair = gm.make_pair(0, 1, pr.F, d, pr.p, pr.q)
        n_a = sc.images[pr.a].n
        for q0, qn in [(0, n_a), (17, 301), (n_a - 1, 1), (5, 0)]:
            off_ref, cand_ref = ctx.band_candidates(pair, q0, qn)
            for _ in range(2):   # two calls in a row: the scratch must be cleared each time
                off, cand, n = _static(gm, ctx, pair, q0, qn, int(off_ref[-1]) + 8)
                np.testing.assert_array_equal(off, off_ref)
                np.testing.assert_array_equal(cand, cand_ref)
                assert n == off_ref[-1]


def test_static_errors(gm, two_view_scene):
    import torch
    sc = two_view_scene
    pr = sc.pairs[0]
    rng = np.random.default_rng(3)
    nb = 40000                                     # 1250 bitmap words per query
    big = scenes.Image(1600, 1200, np.stack([rng.uniform(0, 1599, nb), rng.uniform(0, 1199, nb)], 1).astype(np.float32),
                       np.ones(nb, np.float32), rng.integers(0, 256, (nb, 128), dtype=np.uint8),
                       np.full(nb, -1, np.int32))
    with gm.Context(device=0) as ctx:
        ctx.put_image(0, sc.images[pr.a])
        ctx.put_image(1, big)
        pair = gm.make_pair(0, 1, pr.F, 4.0)
        # 1000 queries x 1250 words x 4 bytes = 5 MB > the 4 MiB scratch: rejected with a clear error
        with pytest.raises(gm.GeomatchError) as e:
            _static(gm, ctx, pair, 0, 1000, 1 << 20)
        assert e.value.status == gm.GM_ERR_INVALID and "scratch" in str(e.value)
        # within the limit it works and equals the allocating entry point
        off_ref, cand_ref = ctx.band_candidates(pair, 0, 500)
        off, cand, _ = _static(gm, ctx, pair, 0, 500, int(off_ref[-1]))
        np.testing.assert_array_equal(off, off_ref)
        np.testing.assert_array_equal(cand, cand_ref)
        # host output buffers are refused (the call would need a staging allocation)
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_band_candidates_static(ctx.h, pair, 0, 10, np.zeros(11, np.int64), np.zeros(100, np.int32), 100)
        assert e.value.status == gm.GM_ERR_INVALID
        # cap too small: GM_ERR_NOMEM with the required size, offsets still written
        if off_ref[-1] > 0:
            off_d = torch.zeros(501, dtype=torch.int64, device="cuda:0")
            cand_d = torch.zeros(1, dtype=torch.int32, device="cuda:0")
            with pytest.raises(gm.GeomatchError) as e:
                gm.gm_band_candidates_static(ctx.h, pair, 0, 500, off_d, cand_d, 0)
            assert e.value.status == gm.GM_ERR_NOMEM and e.value.required == off_ref[-1]
            np.testing.assert_array_equal(off_d.cpu().numpy(), off_ref)


def test_static_allocates_nothing(gm, two_view_scene):
    """Across two calls on a fresh context: the device's free memory and the context's work bytes do not move."""
    import torch
    sc = two_view_scene
    pr = sc.pairs[0]
    n_a = sc.images[pr.a].n
    # first launches of the kernels (module loading) happen here, in a throw-away context
    with gm.Context(device=0) as warm:
        warm.put_image(0, sc.images[pr.a])
        warm.put_image(1, sc.images[pr.b])
        pair = gm.make_pair(0, 1, pr.F, 4.0, pr.p, pr.q)
        off_ref, cand_ref = warm.band_candidates(pair, 0, n_a)
        _static(gm, warm, pair, 0, n_a, int(off_ref[-1]))
    cap = int(off_ref[-1])
    off = torch.zeros(n_a + 1, dtype=torch.int64, device="cuda:0")
    cand = torch.zeros(cap, dtype=torch.int32, device="cuda:0")
    with gm.Context(device=0) as ctx:
        ctx.put_image(0, sc.images[pr.a])
        ctx.put_image(1, sc.images[pr.b])
        torch.cuda.synchronize()
        work0 = gm.gm_image_cache_stats(ctx.h)["work_bytes"]
        free0 = torch.cuda.mem_get_info(0)[0]
        for _ in range(2):
            n = gm.gm_band_candidates_static(ctx.h, pair, 0, n_a, off, cand, cap)
            torch.cuda.synchronize()
            assert gm.gm_image_cache_stats(ctx.h)["work_bytes"] == work0
            assert torch.cuda.mem_get_info(0)[0] == free0
            assert n == cap
            np.testing.assert_array_equal(off.cpu().numpy(), off_ref)
            np.testing.assert_array_equal(cand.cpu().numpy(), cand_ref)


def test_static_under_a_full_budget(gm, two_view_scene):
    """A context whose budget holds its images and nothing more: gm_band_candidates cannot grow its workspace
    (GM_ERR_BUDGET), gm_band_candidates_static still answers, and equals the allocating call of another context."""
    sc = two_view_scene
    pr = sc.pairs[0]
    n_a = sc.images[pr.a].n
    pair = gm.make_pair(0, 1, pr.F, 4.0, pr.p, pr.q)
    with gm.Context(device=0) as ref:
        ref.put_image(0, sc.images[pr.a])
        ref.put_image(1, sc.images[pr.b])
        used = gm.gm_image_cache_stats(ref.h)
        off_ref, cand_ref = ref.band_candidates(pair, 0, n_a)
    budget = used["bytes"] + used["work_bytes"]
    with gm.Context(device=0, mem_budget_bytes=budget) as ctx:
        ctx.put_image(0, sc.images[pr.a])
        ctx.put_image(1, sc.images[pr.b])
        with pytest.raises(gm.GeomatchError) as e:
            ctx.band_candidates(pair, 0, n_a)
        assert e.value.status == gm.GM_ERR_BUDGET
        for _ in range(2):
            off, cand, n = _static(gm, ctx, pair, 0, n_a, int(off_ref[-1]))
            np.testing.assert_array_equal(off, off_ref)
            np.testing.assert_array_equal(cand, cand_ref)
            assert n == off_ref[-1]


def test_static_refuses_host_page_locked_outputs(gm, two_view_scene):
    """Page-locked host memory is not device memory of the context's device: refused before any launch."""
    import torch
    sc = two_view_scene
    pr = sc.pairs[0]
    with gm.Context(device=0) as ctx:
        ctx.put_image(0, sc.images[pr.a])
        ctx.put_image(1, sc.images[pr.b])
        pair = gm.make_pair(0, 1, pr.F, 4.0, pr.p, pr.q)
        off = torch.zeros(11, dtype=torch.int64).pin_memory()
        cand = torch.zeros(100, dtype=torch.int32).pin_memory()
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_band_candidates_static(ctx.h, pair, 0, 10, off, cand, 100)
        assert e.value.status == gm.GM_ERR_INVALID and "device memory" in str(e.value)
