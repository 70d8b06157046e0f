"""Bit-exact parity at full size, in the launch configuration bench.py times (the whole batch in one call, CUDA
graph replay), on sampled pairs the oracle computes one by one (Sec. 6.2, Eqs. 2-3; App. A Step 4).

* The dense scene: street geometry, 1000 images of 16000 keypoints, the top pairs by co-visibility, at every band
  d = 2, 4, 8, 16 px and the whole-image band (exhaustive matching).  A 48 px band gives query groups whose
  candidate streams are longer than a group stages in shared memory (those positions are read from global memory),
  and a candidate-stream buffer far too small for the batch forces the grow-and-rerun path.
* The street component: 1000 images of 2000-20000 keypoints, about 18600 pairs with d in [2, 8] px per pair,
  autotuned, every path against the oracle on sampled pairs.
"""
import math

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu

N_SAMPLE = 24            # sampled pairs per band (the oracle compares each one in full)
N_SAMPLE_INF = 20        # sampled pairs of the whole-image band


@pytest.fixture(scope="module")
def gm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06235_gb300 import geomatch
    geomatch.load_library()
    return geomatch


@pytest.fixture(scope="module")
def dense(gm):
    import torch
    sc = scenes.street(n_kp=16000, n_pairs=30000)
    ctx = gm.Context(device=0, stream=torch.cuda.current_stream())
    ctx.put_images({k: im for k, im in enumerate(sc.images)})
    ctx.set_option(gm.GM_OPT_GRAPH, 1)
    sample = np.sort(np.random.default_rng(1512).choice(len(sc.pairs), N_SAMPLE, replace=False))
    yield sc, ctx, sample
    ctx.close()


def _with_d(pairs, d):
    return [scenes.Pair(p.a, p.b, p.F, d, p.p, p.q) for p in pairs]


def _batch(gm, ctx, sc, pairs, reps=3):
    """gm_match_pairs over `pairs` as bench.py calls it (device outputs); the last of `reps` calls is returned
    (with graph replay on, the first call runs directly, the second captures, the third replays)."""
    import torch
    gp = gm.make_pairs([p.a for p in pairs], [p.b for p in pairs],
                       np.stack([np.asarray(p.F, np.float32).reshape(9) for p in pairs]), [p.d for p in pairs],
                       [p.p for p in pairs], [p.q for p in pairs])
    cap = sum(sc.images[p.a].n for p in pairs)
    off = torch.empty(len(pairs) + 1, dtype=torch.int64, device="cuda:0")
    rows = torch.empty((max(cap, 1), 2), dtype=torch.int32, device="cuda:0")
    for _ in range(reps):
        n = gm.gm_match_pairs(ctx.h, gp, off, rows, cap)
    torch.cuda.synchronize()
    return off.cpu().numpy(), rows[:n], ctx.stats()


def _pair_rows(off, rows, k):
    return rows[int(off[k]):int(off[k + 1])].cpu().numpy()


@pytest.mark.parametrize("d", [2.0, 4.0, 8.0, 16.0])
def test_dense_sampled_pairs_bit_exact(gm, dense, d):
    sc, ctx, sample = dense
    pairs = _with_d(sc.pairs, d)
    off, rows, st = _batch(gm, ctx, sc, pairs)
    assert st["n_device_errors"] == 0 and st["path_used"] == gm.GM_PATH_TC
    sub = [pairs[k] for k in sample]
    want, ncs = oracle.match_batch(sc.images, sub)
    for k, mj in zip(sample, want):
        np.testing.assert_array_equal(_pair_rows(off, rows, k), oracle.matches_from_match_j(mj),
                                      err_msg=f"d = {d}, pair {k}")
    # the sampled pairs as a batch of their own: the same rows, and sum |C_i| equal to the oracle's
    off_s, rows_s, st_s = _batch(gm, ctx, sc, sub, reps=1)
    assert st_s["n_candidates"] == int(ncs.sum())
    for t, k in enumerate(sample):
        np.testing.assert_array_equal(_pair_rows(off_s, rows_s, t), _pair_rows(off, rows, k))


def test_dense_long_streams_bit_exact(gm, dense):
    """d = 48 px on the sampled pairs (one batch): a group's candidate stream is then longer than the positions it
    stages in shared memory (about 1200 against 1024 at 16000 keypoints), so the matcher reads them from global
    memory; the rows stay exactly the oracle's."""
    sc, ctx, sample = dense
    sub = _with_d([sc.pairs[k] for k in sample], 48.0)
    off, rows, st = _batch(gm, ctx, sc, sub)
    assert st["n_device_errors"] == 0 and st["n_unstaged_groups"] > 0
    want, ncs = oracle.match_batch(sc.images, sub)
    assert st["n_candidates"] == int(ncs.sum())
    for t, mj in enumerate(want):
        np.testing.assert_array_equal(_pair_rows(off, rows, t), oracle.matches_from_match_j(mj),
                                      err_msg=f"d = 48, pair {t}")


def test_dense_whole_image_band_bit_exact(gm, dense):
    """d = inf on the first 300 pairs (the bench's exhaustive leg): 20 sampled pairs in full against the oracle's
    exhaustive search (16000 queries x 16000 targets each)."""
    sc, ctx, _ = dense
    pairs = _with_d(sc.pairs[:300], math.inf)
    off, rows, st = _batch(gm, ctx, sc, pairs)
    assert st["n_device_errors"] == 0
    assert st["n_candidates"] == sum(sc.images[p.a].n * sc.images[p.b].n for p in pairs)
    sample = np.sort(np.random.default_rng(1513).choice(len(pairs), N_SAMPLE_INF, replace=False))
    want, ncs = oracle.match_batch(sc.images, [pairs[k] for k in sample])
    for k, mj, nc in zip(sample, want, ncs):
        assert nc == sc.images[pairs[k].a].n * sc.images[pairs[k].b].n
        np.testing.assert_array_equal(_pair_rows(off, rows, k), oracle.matches_from_match_j(mj),
                                      err_msg=f"d = inf, pair {k}")


def test_dense_stream_overflow_rerun(gm, dense):
    """A candidate-stream buffer of 4096 entries for the sampled pairs at d = 16: the batch overflows, the buffer
    grows to what it needed and the batch runs again, with the same rows as a context that never overflowed."""
    import torch
    sc, ctx, sample = dense
    sub = _with_d([sc.pairs[k] for k in sample], 16.0)
    off_r, rows_r, st_r = _batch(gm, ctx, sc, sub, reps=1)
    with gm.Context(device=0, stream=torch.cuda.current_stream()) as small:
        small.set_option(gm.GM_OPT_STREAM_CAP, 4096)
        used = sorted({p.a for p in sub} | {p.b for p in sub})
        small.put_images({k: sc.images[k] for k in used})
        off, rows, st = _batch(gm, small, sc, sub, reps=1)
    assert st["n_stream_reruns"] >= 1 and st_r["n_stream_reruns"] == 0
    assert st["n_candidates"] == st_r["n_candidates"]
    np.testing.assert_array_equal(off, off_r)
    np.testing.assert_array_equal(rows.cpu().numpy(), rows_r.cpu().numpy())


def test_street_full_batch_sampled_bit_exact(gm):
    """The whole street batch in one call, autotuned, with graph replay: 50 sampled pairs exactly as the oracle,
    and the mma.sync and dp4a paths give the same rows over the whole batch."""
    import torch
    sc = scenes.street()
    with gm.Context(device=0, stream=torch.cuda.current_stream()) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        ctx.autotune(sc.pairs, repeats=1)
        ctx.set_option(gm.GM_OPT_GRAPH, 1)
        off, rows, st = _batch(gm, ctx, sc, sc.pairs)
        assert st["n_device_errors"] == 0
        sample = np.sort(np.random.default_rng(1514).choice(len(sc.pairs), 50, replace=False))
        want, ncs = oracle.match_batch(sc.images, [sc.pairs[k] for k in sample])
        for k, mj in zip(sample, want):
            np.testing.assert_array_equal(_pair_rows(off, rows, k), oracle.matches_from_match_j(mj),
                                          err_msg=f"street pair {k}")
        ref = rows.cpu().numpy()
        for path, group in ((gm.GM_PATH_MMA, 16), (gm.GM_PATH_SIMT, 16)):
            ctx.set_option(gm.GM_OPT_PATH, path)
            ctx.set_option(gm.GM_OPT_MMA_GROUP, group)
            off2, rows2, st2 = _batch(gm, ctx, sc, sc.pairs, reps=1)
            assert st2["n_candidates"] == st["n_candidates"]
            np.testing.assert_array_equal(off2, off)
            np.testing.assert_array_equal(rows2.cpu().numpy(), ref)
