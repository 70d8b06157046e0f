"""The device-side failure path: a bounded wait that runs out is reported as GM_ERR_TIMEOUT and leaves the context
usable (the wait is on a flag that nothing sets; no trap, no fault, no hang)."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06235_gb300 import geomatch
    geomatch.load_library()
    return geomatch


def test_bounded_wait_times_out_and_context_survives(gm, two_view_scene):
    sc = two_view_scene
    with gm.Context(device=0) as ctx:
        assert gm.gm_selftest_wait(ctx.h, 2000, True) == gm.GM_OK
        t0 = time.perf_counter()
        assert gm.gm_selftest_wait(ctx.h, 20000, False) == gm.GM_ERR_TIMEOUT
        assert 0.015 < time.perf_counter() - t0 < 2.0
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_selftest_wait(ctx.h, 0, False)
        assert e.value.status == gm.GM_ERR_INVALID
        # the context still matches, and as before
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m = ctx.match_pairs(sc.pairs)
        assert off[-1] > 500
        assert gm.gm_selftest_wait(ctx.h, 2000, True) == gm.GM_OK
        off2, m2 = ctx.match_pairs(sc.pairs)
        np.testing.assert_array_equal(m, m2)
