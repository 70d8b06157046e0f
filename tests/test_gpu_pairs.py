"""gm_select_pairs (candidate image pairs, Sec. 6.1) against the oracle, through the C ABI: identical rows, from a
handful of cameras to 6000 (street-like visibility: every point seen by a run of neighbouring cameras)."""
import numpy as np
import pytest

import scenes
from oracle import pairs as op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06235_gb300 import geomatch
    geomatch.load_library()
    return geomatch


def _random_visibility(rng, n_cams, n_points, max_deg):
    deg = rng.integers(0, max_deg + 1, n_points)
    off = np.zeros(n_points + 1, np.int64)
    off[1:] = np.cumsum(np.minimum(deg, n_cams))
    cams = np.concatenate([np.sort(rng.choice(n_cams, min(d, n_cams), replace=False)) for d in deg]
                          + [np.zeros(0, np.int64)]).astype(np.int32)
    return off, cams


@pytest.mark.parametrize("n_cams,n_points,max_deg", [(1, 10, 3), (5, 40, 4), (40, 3000, 8), (700, 20000, 40)])
@pytest.mark.parametrize("T,k", [(-1, 3), (0, 1), (2, 5), (8, 10000)])
def test_random_visibility(gm, n_cams, n_points, max_deg, T, k):
    rng = np.random.default_rng(n_cams * 7 + n_points + T + k)
    off, cams = _random_visibility(rng, n_cams, n_points, max_deg)
    with gm.Context(device=0) as ctx:
        got = ctx.select_pairs(n_cams, off, cams, T, k)
    want = op.select_pairs(n_cams, off, cams, T, k)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("k", [3, 10, 1000])
def test_facade_visibility(gm, facade_scene, k):
    off, cams, n_cams = scenes.visibility(facade_scene)
    with gm.Context(device=0) as ctx:
        got = ctx.select_pairs(n_cams, off, cams, 8, k)
    np.testing.assert_array_equal(got, op.select_pairs(n_cams, off, cams, 8, k))


def test_device_inputs_outputs_and_errors(gm):
    import torch
    rng = np.random.default_rng(4)
    off, cams = _random_visibility(rng, 30, 2000, 6)
    want = op.select_pairs(30, off, cams, 1, 4)
    with gm.Context(device=0) as ctx:
        out = torch.zeros((len(want) + 5, 3), dtype=torch.int32, device="cuda:0")
        n = gm.gm_select_pairs(ctx.h, 30, torch.from_numpy(off).cuda(), torch.from_numpy(cams).cuda(), 1, 4, out,
                               out.shape[0])
        np.testing.assert_array_equal(out[:n].cpu().numpy(), want)
        with pytest.raises(gm.GeomatchError) as e:   # cap too small: the required size comes back
            gm.gm_select_pairs(ctx.h, 30, off, cams, 1, 4, np.zeros((1, 3), np.int32), 1)
        assert e.value.status == gm.GM_ERR_NOMEM and e.value.required == len(want)
        bad = cams.copy()
        j = int(np.argmax(np.diff(off) >= 2))
        bad[off[j] + 1] = bad[off[j]]   # a point listing one camera twice
        with pytest.raises(gm.GeomatchError) as e:
            ctx.select_pairs(30, off, bad, 1, 4)
        assert e.value.status == gm.GM_ERR_INVALID
        with pytest.raises(gm.GeomatchError) as e:
            ctx.select_pairs(49153, off, cams, 1, 4)
        assert e.value.status == gm.GM_ERR_INVALID


@pytest.mark.parametrize("T,k", [(8, 600), (20, 3), (-1, 2)])
def test_six_thousand_cameras(gm, T, k):
    off, cams, _ = scenes.path_visibility(6000, 300000, seed=6000 + k)
    with gm.Context(device=0) as ctx:
        got = ctx.select_pairs(6000, off, cams, T, k)
    want = op.select_pairs(6000, off, cams, T, k)
    assert len(want) >= 5000   # every query chose at least its neighbours
    np.testing.assert_array_equal(got, want)


def test_wide_camera_range_and_bad_ids(gm):
    """30000 cameras of which only the first 900 see points: the transpose takes its global-memory path (too many
    cameras for a block-local histogram) and every row is 30000 counts wide, yet with T >= 0 the idle cameras are
    never candidates, so the rows equal the oracle's over the 900 cameras.  A camera id past n_cams is an error."""
    off, cams, _ = scenes.path_visibility(900, 60000, seed=77)
    want = op.select_pairs(900, off, cams, 3, 40)
    with gm.Context(device=0) as ctx:
        np.testing.assert_array_equal(ctx.select_pairs(30000, off, cams, 3, 40), want)
        np.testing.assert_array_equal(ctx.select_pairs(900, off, cams, 3, 40), want)
        bad = cams.copy()
        bad[len(bad) // 2] = 900
        with pytest.raises(gm.GeomatchError) as e:
            ctx.select_pairs(900, off, bad, 3, 40)
        assert e.value.status == gm.GM_ERR_INVALID
