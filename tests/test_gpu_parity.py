"""GPU path vs the CPU oracle, through the C ABI (bit-exact: match lists and candidate sets are integers).

Sizes span several grid cells, work items and ragged tails; the full-size batch (1200 facade pairs of 8000
keypoints, the benchmark's launch configuration) is checked on a sample of pairs that the oracle computes one
by one, plus schedule / cell-size / path invariance over the whole batch.
"""
import math

import numpy as np
import pytest

import oracle
import scenes
from tests import golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06235_gb300 import geomatch
    geomatch.load_library()
    return geomatch


def _oracle_rows(sc, pr):
    A, B = sc.images[pr.a], sc.images[pr.b]
    mj, nc = oracle.match_pair(A.xy, A.desc, B.xy, B.desc, pr.F, pr.d, pr.p, pr.q)
    return oracle.matches_from_match_j(mj), nc


PATHS = [("tc", 1, 16), ("simt", 3, 16), ("mma16", 2, 16), ("mma32", 2, 32)]


def _gpu_rows(gm, sc, pairs=None, cell_px=0, path=0, schedule=0, group=16):
    pairs = sc.pairs if pairs is None else pairs
    with gm.Context(device=0, cell_px=cell_px, path=path) as ctx:
        if schedule:
            ctx.set_option(gm.GM_OPT_SCHEDULE, schedule)
        if group != 16:
            ctx.set_option(gm.GM_OPT_MMA_GROUP, group)
        used = sorted({p.a for p in pairs} | {p.b for p in pairs})
        for k in used:
            ctx.put_image(k, sc.images[k])
        off, m = ctx.match_pairs(pairs)
        st = ctx.stats()
    return gm.split_matches(off, m), st


@pytest.mark.parametrize("path", PATHS, ids=lambda p: p[0])
def test_two_view_bit_exact(gm, two_view_scene, path):
    sc = two_view_scene
    rows, st = _gpu_rows(gm, sc, path=path[1], group=path[2])
    want, nc = _oracle_rows(sc, sc.pairs[0])
    np.testing.assert_array_equal(rows[0], want)
    assert st["n_candidates"] == nc
    assert st["n_examined"] >= nc


@pytest.mark.parametrize("path", PATHS, ids=lambda p: p[0])
@pytest.mark.parametrize("cell_px", [4, 8, 16, 64, 128])
def test_two_view_cell_sizes(gm, two_view_scene, cell_px, path):
    sc = two_view_scene
    rows, st = _gpu_rows(gm, sc, cell_px=cell_px, path=path[1], group=path[2])
    want, nc = _oracle_rows(sc, sc.pairs[0])
    np.testing.assert_array_equal(rows[0], want)
    assert st["n_candidates"] == nc


def _random_batch(seeds, d_values, levels=256, n_a=300, n_b=411):
    """One scene per (seed, d): several pairs of generic geometry in one batch (images renumbered)."""
    images, pairs = [], []
    for s in seeds:
        for d in d_values:
            sc = scenes.random_small(s, n_a, n_b, d=d, desc_levels=levels)
            a, b = len(images), len(images) + 1
            images += sc.images
            pr = sc.pairs[0]
            pairs.append(scenes.Pair(a, b, pr.F, d, 4, 5))
            pairs.append(scenes.Pair(b, a, pr.F.reshape(3, 3).T.copy().reshape(9), d, 9, 10))
    return scenes.Scene("random_batch", images, pairs)


@pytest.mark.parametrize("path", PATHS, ids=lambda p: p[0])
@pytest.mark.parametrize("levels", [256, 4, 2])
def test_random_pairs_batched(gm, levels, path):
    sc = _random_batch(range(3), [0.0, 1.5, 4.0, 13.0, math.inf], levels=levels)
    rows, st = _gpu_rows(gm, sc, path=path[1], group=path[2])
    total = 0
    for k, pr in enumerate(sc.pairs):
        want, nc = _oracle_rows(sc, pr)
        np.testing.assert_array_equal(rows[k], want, err_msg=f"pair {k} d={pr.d}")
        total += nc
    assert st["n_candidates"] == total


def test_band_candidates_equal_linear_search(gm):
    """The cell walk + exact test returns exactly Eq. 2's set (linear search) for every query: steep, shallow and
    oblique lines, several band widths."""
    sc = _random_batch(range(2), [0.5, 4.0, 25.0], n_a=120, n_b=700)
    with gm.Context(device=0) as ctx:
        for k, im in enumerate(sc.images):
            ctx.put_image(k, im)
        for pr in sc.pairs:
            off, cand = ctx.band_candidates(gm.make_pair(pr.a, pr.b, pr.F, pr.d, pr.p, pr.q))
            A, B = sc.images[pr.a], sc.images[pr.b]
            for i in range(A.n):
                want = oracle.band_set(pr.F, pr.d, A.xy[i, 0], A.xy[i, 1], B.xy)
                np.testing.assert_array_equal(cand[off[i]:off[i + 1]], want)


@pytest.mark.parametrize("case", golden.band_cases(), ids=lambda c: c["name"])
def test_band_golden_on_gpu(gm, case):
    W, H = 2048, 2048
    pts = case["points"]
    qxy = np.array([case["q"]], np.float32)
    with gm.Context(device=0) as ctx:
        ctx.put_image(0, width=W, height=H, xy=qxy, scale=None, desc=np.zeros((1, 128), np.uint8))
        ctx.put_image(1, width=W, height=H, xy=pts, scale=None, desc=np.zeros((len(pts), 128), np.uint8))
        off, cand = ctx.band_candidates(gm.make_pair(0, 1, case["F"], case["d"]))
    np.testing.assert_array_equal(cand, np.nonzero(case["expected"])[0])


@pytest.mark.parametrize("path", PATHS, ids=lambda p: p[0])
@pytest.mark.parametrize("case", golden.ratio_cases(), ids=lambda c: c["name"])
def test_ratio_golden_on_gpu(gm, case, path):
    n = case["bd"].shape[0]
    with gm.Context(device=0, path=path[1]) as ctx:
        ctx.put_image(0, width=64, height=64, xy=np.array([[5.0, 5.0]], np.float32), scale=None,
                      desc=case["qd"][None])
        ctx.put_image(1, width=64, height=64, xy=np.full((n, 2), 10.0, np.float32).reshape(-1, 2), scale=None,
                      desc=case["bd"].reshape(-1, 128))
        off, m = ctx.match_pairs([gm.make_pair(0, 1, np.eye(3).reshape(9), math.inf, case["p"], case["q"])])
    want = [] if case["expected"] < 0 else [[0, case["expected"]]]
    np.testing.assert_array_equal(m.reshape(-1, 2), np.array(want, np.int32).reshape(-1, 2))


@pytest.mark.parametrize("path", PATHS, ids=lambda p: p[0])
def test_edge_cases(gm, path):
    rng = np.random.default_rng(5)
    W, H = 640, 480
    xy = np.stack([rng.uniform(0, W, 500), rng.uniform(0, H, 500)], 1).astype(np.float32)
    xy[:40] = np.array([[np.float32(k * 16), np.float32(32)] for k in range(40)], np.float32)  # on cell borders
    xy[40:60] = [W - 1e-3, H - 1e-3]                                                            # one corner cell
    xy[60:70] = [0.0, 0.0]
    desc = rng.integers(0, 256, (500, 128), dtype=np.uint8)
    desc[100:110] = desc[200]                                                                   # duplicates
    empty = np.zeros((0, 2), np.float32)
    F_gen = scenes.random_small(9, 4, 4, w=W, h=H).pairs[0].F
    F_vert = np.array([0, 0, 1, 0, 0, 0, 0, 0, -300], np.float32)        # lines x' = 300 (pure column)
    F_zero = np.array([0, 0, 0, 0, 0, 0, 0, 0, 1], np.float32)          # no line at all
    images = [scenes.Image(W, H, xy, np.ones(500, np.float32), desc, np.full(500, -1, np.int32)),
              scenes.Image(W, H, empty, np.zeros(0, np.float32), np.zeros((0, 128), np.uint8), np.zeros(0, np.int32)),
              scenes.Image(W, H, xy[:1].copy(), np.ones(1, np.float32), desc[:1].copy(), np.full(1, -1, np.int32))]
    pairs = [scenes.Pair(0, 0, F_gen, 6.0), scenes.Pair(0, 1, F_gen, 6.0), scenes.Pair(1, 0, F_gen, 6.0),
             scenes.Pair(0, 2, F_gen, math.inf), scenes.Pair(0, 0, scenes.RECTIFIED_F, 0.0),
             scenes.Pair(0, 0, F_vert, 3.0), scenes.Pair(0, 0, F_zero, 5.0), scenes.Pair(0, 0, F_zero, math.inf),
             scenes.Pair(2, 0, F_gen, 1e6)]
    sc = scenes.Scene("edges", images, pairs)
    rows, _ = _gpu_rows(gm, sc, path=path[1], group=path[2])
    for k, pr in enumerate(pairs):
        want, _ = _oracle_rows(sc, pr)
        np.testing.assert_array_equal(rows[k], want, err_msg=f"pair {k}")


def test_invalid_inputs(gm):
    with gm.Context(device=0) as ctx:
        with pytest.raises(gm.GeomatchError) as e:
            ctx.put_image(0, width=10, height=10, xy=np.array([[10.0, 1.0]], np.float32), scale=None,
                          desc=np.zeros((1, 128), np.uint8))
        assert e.value.status == gm.GM_ERR_INVALID
        ctx.put_image(0, width=10, height=10, xy=np.array([[1.0, 1.0], [2.0, 2.0]], np.float32), scale=None,
                      desc=np.zeros((2, 128), np.uint8))
        with pytest.raises(gm.GeomatchError) as e:
            ctx.match_pairs([gm.make_pair(0, 7, np.eye(3).reshape(9), 1.0)])
        assert e.value.status == gm.GM_ERR_NOT_FOUND
        with pytest.raises(gm.GeomatchError) as e:
            ctx.match_pairs([gm.make_pair(0, 0, np.eye(3).reshape(9), 1.0, 5, 5)])
        assert e.value.status == gm.GM_ERR_INVALID
        with pytest.raises(gm.GeomatchError) as e:
            ctx.match_pairs([gm.make_pair(0, 0, np.eye(3).reshape(9), float("nan"))])
        assert e.value.status == gm.GM_ERR_INVALID
        off = np.zeros(2, np.int64)
        m = np.zeros((1, 2), np.int32)
        F = np.eye(3, dtype=np.float32).reshape(9)
        n = gm.gm_match_pairs(ctx.h, [gm.make_pair(0, 0, F, math.inf, 1, 2)], off, m, 0)
        assert n == 0


def test_facade_full_batch_sampled(gm, facade_scene):
    """Full-size batch in the benchmark's launch configuration; 24 pairs spread over it checked exactly; the other
    paths and the per-pair launch schedule give identical lists over the whole batch."""
    sc = facade_scene
    rows, st = _gpu_rows(gm, sc)
    sample = list(range(0, len(sc.pairs), 50))
    wants = oracle.match_batch(sc.images, [sc.pairs[k] for k in sample])[0]
    for k, mj in zip(sample, wants):
        np.testing.assert_array_equal(rows[k], oracle.matches_from_match_j(mj), err_msg=f"pair {k}")
    assert st["n_pairs"] == len(sc.pairs)
    assert st["n_matches"] == sum(len(r) for r in rows)
    # per-pair launches (plain form) give the same lists over the whole batch
    rows1, st1 = _gpu_rows(gm, sc, schedule=1)
    for k in range(len(sc.pairs)):
        np.testing.assert_array_equal(rows1[k], rows[k])
    assert st1["n_candidates"] == st["n_candidates"]
    for name, path, group in PATHS:
        rows2, st2 = _gpu_rows(gm, sc, path=path, group=group)
        assert st2["n_candidates"] == st["n_candidates"], name
        for k in range(len(sc.pairs)):
            np.testing.assert_array_equal(rows2[k], rows[k], err_msg=f"{name} pair {k}")


def test_graph_replay_equal(gm, facade_scene):
    """GM_OPT_GRAPH: a batch shape seen twice is captured, then replayed; every call gives the direct run's lists,
    also when the pinned pair table changes between replays (same shape, different pairs)."""
    sc = facade_scene
    pairs_a, pairs_b = sc.pairs[:60], sc.pairs[60:120]
    ref_a, st_a = _gpu_rows(gm, sc, pairs=pairs_a)
    ref_b, _ = _gpu_rows(gm, sc, pairs=pairs_b)
    with gm.Context(device=0) as ctx:
        ctx.set_option(gm.GM_OPT_GRAPH, 1)
        for k in sorted({p.a for p in sc.pairs[:120]} | {p.b for p in sc.pairs[:120]}):
            ctx.put_image(k, sc.images[k])
        for it in range(4):
            off, m = ctx.match_pairs(pairs_a)
            got = gm.split_matches(off, m)
            for k in range(len(pairs_a)):
                np.testing.assert_array_equal(got[k], ref_a[k], err_msg=f"call {it} pair {k}")
            assert ctx.stats()["n_candidates"] == st_a["n_candidates"]
        same_shape = sum(sc.images[p.a].n for p in pairs_b) == sum(sc.images[p.a].n for p in pairs_a)
        off, m = ctx.match_pairs(pairs_b)
        got = gm.split_matches(off, m)
        for k in range(len(pairs_b)):
            np.testing.assert_array_equal(got[k], ref_b[k], err_msg=f"second batch pair {k} (same shape {same_shape})")


def test_autotune_and_cache(gm, facade_scene, tmp_path):
    """gm_autotune leaves a valid setting whose lists equal the default run's; the cache file gives the same
    setting back without timing."""
    sc = facade_scene
    pairs = sc.pairs[:24]
    ref, _ = _gpu_rows(gm, sc, pairs=pairs)
    cache = str(tmp_path / "tune.txt")
    used = sorted({p.a for p in pairs} | {p.b for p in pairs})
    with gm.Context(device=0, tuner_cache=cache) as ctx:
        for k in used:
            ctx.put_image(k, sc.images[k])
        r = ctx.autotune(pairs, repeats=1)
        assert r["from_cache"] == 0 and r["cell_px"] in (4, 8, 16) and r["mma_group"] in (16, 32)
        assert r["path"] in (gm.GM_PATH_TC, gm.GM_PATH_MMA, gm.GM_PATH_SIMT) and r["ms"] > 0
        off, m = ctx.match_pairs(pairs)
        got = gm.split_matches(off, m)
        for k in range(len(pairs)):
            np.testing.assert_array_equal(got[k], ref[k])
    with gm.Context(device=0, tuner_cache=cache) as ctx:
        for k in used:
            ctx.put_image(k, sc.images[k])
        r2 = ctx.autotune(pairs, repeats=1)
        assert r2["from_cache"] == 1
        assert (r2["path"], r2["mma_group"], r2["cell_px"]) == (r["path"], r["mma_group"], r["cell_px"])
        off, m = ctx.match_pairs(pairs)
        got = gm.split_matches(off, m)
        for k in range(len(pairs)):
            np.testing.assert_array_equal(got[k], ref[k])


def test_images_put_batch_equals_single_puts(gm, facade_scene):
    """gm_images_put (pageable host arrays, device tensors, page-locked host tensors read in place) registers the same
    images as gm_image_put one by one, scales included; an out-of-image keypoint in any image of a batch is rejected
    and leaves the registered images as they were."""
    import torch
    from oracle import coarse as oc
    sc = facade_scene
    pairs = sc.pairs[:30]
    used = sorted({p.a for p in pairs} | {p.b for p in pairs})
    ref, st_ref = _gpu_rows(gm, sc, pairs=pairs)
    for mode in ("host", "device", "pinned"):
        on_device = mode == "device"
        with gm.Context(device=0) as ctx:
            if mode == "host":
                imgs = {k: sc.images[k] for k in used}
            else:
                put = (lambda a: torch.from_numpy(a).cuda()) if on_device else (lambda a: torch.from_numpy(a).pin_memory())
                imgs = {k: scenes.Image(sc.images[k].width, sc.images[k].height, put(sc.images[k].xy),
                                        put(sc.images[k].scale), put(sc.images[k].desc), sc.images[k].pid) for k in used}
            ctx.put_images(imgs)
            off, m = ctx.match_pairs(pairs)
            got = gm.split_matches(off, m)
            for k in range(len(pairs)):
                np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{mode} pair {k}")
            assert ctx.stats()["n_candidates"] == st_ref["n_candidates"]
            for k in used[:3]:   # the scales arrived: the coarse selection equals the oracle's
                for g, w in zip(ctx.coarse_selection(k), oc.select_by_scale(sc.images[k].scale)):
                    np.testing.assert_array_equal(g, w)
            # a bad keypoint in the second image of a new batch: nothing changes
            bad = scenes.Image(sc.images[used[1]].width, sc.images[used[1]].height, sc.images[used[1]].xy.copy(),
                               sc.images[used[1]].scale, sc.images[used[1]].desc, sc.images[used[1]].pid)
            bad.xy[7] = [bad.width + 5.0, 1.0]
            other = scenes.Image(sc.images[used[0]].width, sc.images[used[0]].height, sc.images[used[0]].xy[::-1].copy(),
                                 sc.images[used[0]].scale, sc.images[used[0]].desc[::-1].copy(), sc.images[used[0]].pid)
            with pytest.raises(gm.GeomatchError) as e:
                ctx.put_images({used[0]: other, used[1]: bad})
            assert e.value.status == gm.GM_ERR_INVALID
            off, m = ctx.match_pairs(pairs)
            got = gm.split_matches(off, m)
            for k in range(len(pairs)):
                np.testing.assert_array_equal(got[k], ref[k], err_msg=f"after rejected batch, pair {k}")
    # page-locked descriptors 8 bytes past a 16-byte boundary are staged instead of read in place (same result);
    # device descriptors at such an offset are refused before any kernel reads them
    def shifted(a, device):
        buf = torch.zeros(a.size + 8, dtype=torch.uint8, device=device)
        if device == "cpu":
            buf = buf.pin_memory()
        v = buf[8:].view(a.shape)
        v.copy_(torch.from_numpy(a))
        assert v.data_ptr() % 16 == 8
        return v
    pin = lambda a: torch.from_numpy(a).pin_memory()
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: scenes.Image(sc.images[k].width, sc.images[k].height, pin(sc.images[k].xy),
                                        pin(sc.images[k].scale), shifted(sc.images[k].desc, "cpu"), sc.images[k].pid)
                        for k in used})
        off, m = ctx.match_pairs(pairs)
        got = gm.split_matches(off, m)
        for k in range(len(pairs)):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"unaligned page-locked, pair {k}")
        im = sc.images[used[0]]
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_images_put(ctx.h, [(999, im.width, im.height, torch.from_numpy(im.xy).cuda(), None,
                                      shifted(im.desc, "cuda:0"))])
        assert e.value.status == gm.GM_ERR_INVALID
        assert gm.gm_image_info(ctx.h, 999) is None


def test_street_uneven_batch_sampled(gm):
    """Uneven batch (street geometry, 2k-20k keypoints per image, d in [2, 8] per pair) in one call with graph
    replay and the autotuned setting: every 10th pair exactly as the oracle, all paths equal over the batch."""
    sc = scenes.street(n_images=120, n_points=150_000, n_pairs=400)
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        ctx.set_option(gm.GM_OPT_GRAPH, 1)
        ctx.autotune(sc.pairs, repeats=1)
        for _ in range(3):   # direct run, capture, replay
            off, m = ctx.match_pairs(sc.pairs)
        rows = gm.split_matches(off, m)
        st = ctx.stats()
    sample = list(range(0, len(sc.pairs), 10))
    wants = oracle.match_batch(sc.images, [sc.pairs[k] for k in sample])[0]
    for k, mj in zip(sample, wants):
        np.testing.assert_array_equal(rows[k], oracle.matches_from_match_j(mj), err_msg=f"pair {k}")
    for name, path, group in PATHS:
        rows2, st2 = _gpu_rows(gm, sc, path=path, group=group)
        assert st2["n_candidates"] == st["n_candidates"], name
        for k in range(len(sc.pairs)):
            np.testing.assert_array_equal(rows2[k], rows[k], err_msg=f"{name} pair {k}")


def test_stream_buffer_overflow_reruns(gm, facade_scene):
    """A candidate-stream buffer far too small for the batch forces the grow-and-rerun path; results unchanged."""
    sc = facade_scene
    pairs = sc.pairs[:40]
    rows, st = _gpu_rows(gm, sc, pairs=pairs)
    with gm.Context(device=0) as ctx:
        ctx.set_option(gm.GM_OPT_STREAM_CAP, 1000)
        for k in sorted({p.a for p in pairs} | {p.b for p in pairs}):
            ctx.put_image(k, sc.images[k])
        off, m = ctx.match_pairs(pairs)
        st2 = ctx.stats()
    got = gm.split_matches(off, m)
    for k in range(len(pairs)):
        np.testing.assert_array_equal(got[k], rows[k])
    assert st2["n_candidates"] == st["n_candidates"]


def test_serving_alone_equals_mix(gm, facade_scene):
    sc = facade_scene
    pairs = sc.pairs[:60]
    with gm.Context(device=0, max_inflight=3) as ctx:
        for k in sorted({p.a for p in pairs} | {p.b for p in pairs}):
            ctx.put_image(k, sc.images[k])
        off, m = ctx.match_pairs(pairs)
        batch_rows = gm.split_matches(off, m)
        tickets = [ctx.submit(gm.make_pair(p.a, p.b, p.F, p.d, p.p, p.q)) for p in pairs]
        for k, t in enumerate(tickets):
            got, lat = ctx.poll(t, timeout_ms=60000)
            np.testing.assert_array_equal(got, batch_rows[k])
            assert lat > 0
        alone = ctx.submit(gm.make_pair(pairs[7].a, pairs[7].b, pairs[7].F, pairs[7].d))
        got, _ = ctx.poll(alone, timeout_ms=60000)
        np.testing.assert_array_equal(got, batch_rows[7])
        ss = ctx.serving_stats()
        assert ss["completed"] == len(pairs) + 1 and ss["failed"] == 0


@pytest.mark.parametrize("path", PATHS, ids=[p[0] for p in PATHS])
def test_extreme_descriptors_exact(gm, path):
    """Distances at the top of the range (descriptors of 0 and 255 only, D up to 128 * 255^2 < 2^23) decide the
    ratio test exactly: a query of zeros against all-255 (D2 = 8323200) and 81 x 255 + v (D1 = 5267025 + v^2)
    matches for v = 244 (25 D1 = 133164025 < 16 D2 = 133171200) and not for v = 245 (133176250); random 0/255
    descriptors besides, in every band setting, equal the oracle."""
    rng = np.random.default_rng(17)
    W, H = 256, 256
    def img(desc):
        n = len(desc)
        xy = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], 1).astype(np.float32)
        return scenes.Image(W, H, xy, np.ones(n, np.float32), np.asarray(desc, np.uint8), np.full(n, -1, np.int32))
    zeros = np.zeros((4, 128), np.uint8)
    def near(v):
        d = np.zeros(128, np.uint8)
        d[:81] = 255
        d[81] = v
        return d
    full = np.full(128, 255, np.uint8)
    binary = (rng.integers(0, 2, (300, 128)) * 255).astype(np.uint8)
    alt = np.tile(np.array([0, 255], np.uint8), 64)
    images = [img(zeros), img([full, near(244)]), img([full, near(245)]),
              img(np.concatenate([binary, alt[None], alt[::-1][None], zeros[:1], full[None]])),
              img(np.concatenate([binary[::-1], full[None], alt[None]]))]
    F = scenes.random_small(3, 4, 4, w=W, h=H).pairs[0].F
    pairs = [scenes.Pair(0, 1, F, math.inf), scenes.Pair(0, 2, F, math.inf), scenes.Pair(3, 4, F, math.inf),
             scenes.Pair(4, 3, F, math.inf), scenes.Pair(3, 4, F, 20.0)]
    sc = scenes.Scene("extremes", images, pairs)
    rows, _ = _gpu_rows(gm, sc, path=path[1], group=path[2])
    for k, pr in enumerate(pairs):
        want, _ = _oracle_rows(sc, pr)
        np.testing.assert_array_equal(rows[k], want, err_msg=f"pair {k}")
    assert rows[0].shape[0] == 4 and (rows[0][:, 1] == 1).all()   # every zero query picks 81 x 255 + 244
    assert rows[1].shape[0] == 0


def test_tc_pipeline_geometries_equal(gm):
    """The tcgen05 path's three pipeline geometries (GM_OPT_TC_PIPE: 6 chunks / 3 groups / 1024 staged positions,
    8 / 2 / 1024, 4 / 4 / 512) give identical rows; with 16000-keypoint images at d = 16 px, streams longer than 512
    positions are read from global memory by the third.  Every 8th pair is checked against the oracle."""
    sc = scenes.street(n_images=60, n_points=120_000, n_kp=16000, n_pairs=80, d=16.0)
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        got = []
        for pipe in range(3):
            ctx.set_option(gm.GM_OPT_TC_PIPE, pipe)
            off, m = ctx.match_pairs(sc.pairs)
            st = ctx.stats()
            assert st["path_used"] == gm.GM_PATH_TC and st["n_device_errors"] == 0
            got.append((gm.split_matches(off, m), st["n_candidates"]))
        with pytest.raises(gm.GeomatchError):
            ctx.set_option(gm.GM_OPT_TC_PIPE, 3)
    for rows, nc in got[1:]:
        assert nc == got[0][1]
        for k in range(len(sc.pairs)):
            np.testing.assert_array_equal(rows[k], got[0][0][k], err_msg=f"pair {k}")
    sample = list(range(0, len(sc.pairs), 8))
    wants = oracle.match_batch(sc.images, [sc.pairs[k] for k in sample])[0]
    for k, mj in zip(sample, wants):
        np.testing.assert_array_equal(got[0][0][k], oracle.matches_from_match_j(mj), err_msg=f"pair {k}")


@pytest.mark.parametrize("levels", [3, 256])
def test_whole_image_ragged_sizes(gm, levels):
    """A batch in which every pair is at d = inf runs the whole-image kernel (128-candidate chunks, 16 epilogue
    warps of one 32-column block each, the block-maximum test on targets of 4096 keypoints or more).  Targets of
    1, 31, 33, 127, 129, 4095, 4096, 4097 and 6000 keypoints (partial 32-column blocks, partial chunks, both sides
    of the test's threshold) against sources of 1 to 300 queries (partial 128-query groups), with a three-level
    descriptor alphabet (many equal distances) and a full one; every pair's rows equal the oracle's."""
    rng = np.random.default_rng(4096 + levels)
    W, H = 800, 600
    n_b = [1, 31, 33, 127, 129, 4095, 4096, 4097, 6000]
    n_a = [1, 127, 129, 300]
    alphabet = np.array([0, 128, 255], np.uint8) if levels == 3 else np.arange(256, dtype=np.uint8)

    def image(n):
        xy = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], 1).astype(np.float32)
        desc = alphabet[rng.integers(0, len(alphabet), (n, 128))]
        return scenes.Image(W, H, xy, np.ones(n, np.float32), desc, np.full(n, -1, np.int32))

    images = [image(n) for n in n_a] + [image(n) for n in n_b]
    F = scenes.random_small(3, 4, 4, w=W, h=H).pairs[0].F
    pairs = [scenes.Pair(a, len(n_a) + b, F, math.inf, 4, 5) for a in range(len(n_a)) for b in range(len(n_b))]
    sc = scenes.Scene("whole_ragged", images, pairs)
    rows, st = _gpu_rows(gm, sc)
    assert st["path_used"] == gm.GM_PATH_TC and st["n_device_errors"] == 0
    for k, pr in enumerate(pairs):
        want, nc = _oracle_rows(sc, pr)
        np.testing.assert_array_equal(rows[k], want, err_msg=f"pair {k}: {images[pr.a].n} x {images[pr.b].n}")
    assert st["n_candidates"] == sum(images[p.a].n * images[p.b].n for p in pairs)
