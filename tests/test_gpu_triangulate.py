"""gm_triangulate (linear least-squares points of the merged tracks, Sec. 6.2 end) against the oracle, through the
C ABI.  Roots and view counts are integers and must be identical; points are FP64 on both sides but the sums run in
different orders, so each point is compared within a first-order perturbation bound of the normal equations:

    |dX| <= ||M^-1|| * g * ( || |A3|^T |A3| || * |X| + || |A3|^T |a4| || ),   g = 4 (2n + 8) eps,

where |A| bounds the magnitudes that enter the rows (|x| |P3| + |P1|, ...), n is the number of views, the 2n + 8
covers the 2n-term sums and the rounding of the rows and of the 3 x 3 solve, and the factor 4 the two sides.
"""
import numpy as np
import pytest

import scenes
from oracle import tracks as ot
from oracle import triangulate as otri

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def gm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06235_gb300 import geomatch
    geomatch.load_library()
    return geomatch


def _bound(Ps, xys, X):
    Ab = []
    for P, (x, y) in zip(Ps, xys):
        P = np.abs(np.asarray(P, np.float64))
        Ab.append(abs(float(x)) * P[2] + P[0])
        Ab.append(abs(float(y)) * P[2] + P[1])
    Ab = np.array(Ab)
    rows = []
    for P, (x, y) in zip(Ps, xys):
        P = np.asarray(P, np.float64)
        rows += [float(x) * P[2] - P[0], float(y) * P[2] - P[1]]
    A = np.array(rows)
    M = A[:, :3].T @ A[:, :3]
    smin = np.linalg.svd(M, compute_uv=False)[-1]
    g = 4.0 * (2 * len(Ps) + 8) * EPS
    mag = np.linalg.norm(Ab[:, :3].T @ Ab[:, :3], 2) * np.linalg.norm(X) + np.linalg.norm(Ab[:, :3].T @ Ab[:, 3])
    return g * mag / smin


def _check_tracks(images, Ps, labels, X, roots, nv, sample=None, rng=None):
    """Roots and view counts of every track; the points of every track (sample=None: the oracle's
    triangulate_tracks) or of `sample` tracks (the oracle's triangulate, one track at a time)."""
    base = np.concatenate([[0], np.cumsum([im.n for im in images])]).astype(np.int64)
    if sample is None:
        want_roots, want_nv, want_X = otri.triangulate_tracks(Ps, [im.xy for im in images], labels)
    else:
        r, c = np.unique(labels, return_counts=True)   # a track: a component with at least two nodes
        want_roots, want_nv = r[c >= 2], c[c >= 2]
    np.testing.assert_array_equal(roots, want_roots)
    np.testing.assert_array_equal(nv, want_nv)
    order = np.argsort(labels, kind="stable")
    starts = np.searchsorted(labels[order], roots)
    ks = np.arange(roots.size) if sample is None else rng.choice(roots.size, min(sample, roots.size), replace=False)
    worst = 0.0
    for t in ks:
        nodes = order[starts[t]:starts[t] + nv[t]]
        img = np.searchsorted(base, nodes, side="right") - 1
        Pl = [Ps[k] for k in img]
        xy = [images[k].xy[v - base[k]] for k, v in zip(img, nodes)]
        ref = want_X[t] if sample is None else otri.triangulate(Pl, xy)
        if not np.isfinite(ref).all():
            assert np.isnan(X[t]).all()
            continue
        tol = _bound(Pl, xy, ref)
        err = np.linalg.norm(X[t] - ref)
        assert err <= tol, (t, X[t], ref, err, tol)
        worst = max(worst, err / tol)
    return worst


def _scene_tracks(gm, ctx, sc):
    base = np.concatenate([[0], np.cumsum([im.n for im in sc.images])]).astype(np.int64)
    ctx.put_images({k: im for k, im in enumerate(sc.images)})
    off, m = ctx.match_pairs(sc.pairs)
    edges = ot.edges_from_matches(base, sc.pairs, off, m)
    labels = ot.labels(int(base[-1]), edges)
    Ps = [otri.camera_matrix(c) for c in sc.cameras]
    return labels, Ps


def test_small_facade_all_tracks(gm):
    sc = scenes.facade(n_images=12, n_kp=1500, n_points=8000, n_pairs=40, min_covis=20)
    with gm.Context(device=0) as ctx:
        labels, Ps = _scene_tracks(gm, ctx, sc)
        X, roots, nv = ctx.triangulate(list(range(len(sc.images))), np.array(Ps), labels)
    assert roots.size > 100
    _check_tracks(sc.images, Ps, labels, X, roots, nv)


def test_facade_device_buffers(gm, facade_scene):
    """Full facade batch: device P, labels and outputs; roots and view counts of every track, points of a sample."""
    import torch
    sc = facade_scene
    with gm.Context(device=0) as ctx:
        labels, Ps = _scene_tracks(gm, ctx, sc)
        ids = np.arange(len(sc.images), dtype=np.int32)
        cap = int(labels.size)
        X = torch.empty((cap, 3), dtype=torch.float64, device="cuda:0")
        roots = torch.empty(cap, dtype=torch.int64, device="cuda:0")
        nv = torch.empty(cap, dtype=torch.int32, device="cuda:0")
        n = gm.gm_triangulate(ctx.h, ids, torch.from_numpy(np.array(Ps).reshape(-1, 12)).cuda(),
                              torch.from_numpy(labels).cuda(), X, roots, nv, cap)
        X, roots, nv = X[:n].cpu().numpy(), roots[:n].cpu().numpy(), nv[:n].cpu().numpy()
    assert n > 10000
    _check_tracks(sc.images, Ps, labels, X, roots, nv, sample=3000, rng=np.random.default_rng(5))


def test_noise_free_points_recovered(gm):
    """Exact projections of known points: every track's point comes back to the float32 rounding of its pixels."""
    rng = np.random.default_rng(11)
    K = scenes.intrinsics(1000.0, 1280, 960)
    cams = []
    for k in range(6):
        c = np.array([2.0 * k - 5.0, 0.3 * k, -12.0])
        cams.append(scenes.camera_at(K, scenes.look_at(c, [0.0, 0.0, 0.0]), c))
    Xw = rng.uniform([-3, -2, -3], [3, 2, 3], (400, 3))
    images, node_pid = [], []
    for cam in cams:
        uv, z = scenes.project(cam, Xw)
        ok = np.nonzero(scenes.inside(uv, 1280, 960) & (z > 0))[0]
        ok = rng.permutation(ok)
        images.append(scenes.Image(1280, 960, uv[ok].astype(np.float32), np.ones(ok.size, np.float32),
                                   rng.integers(0, 256, (ok.size, 128), dtype=np.uint8), ok.astype(np.int32)))
        node_pid.append(ok)
    pid = np.concatenate(node_pid)
    first = {}
    labels = np.empty(pid.size, np.int64)
    for v, p in enumerate(pid):
        labels[v] = first.setdefault(int(p), v)
    Ps = [otri.camera_matrix(c) for c in cams]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(images)})
        X, roots, nv = ctx.triangulate(list(range(6)), np.array(Ps), labels)
    _check_tracks(images, Ps, labels, X, roots, nv)
    truth = Xw[pid[roots]]
    assert np.abs(X - truth).max() < 2e-3


def test_singular_and_singletons(gm):
    """Cameras whose third row ignores depth make the system exactly singular: NaN on both sides.  Nodes alone in
    their component are not tracks."""
    P = np.array([[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 0, 1.0]])
    im = scenes.Image(64, 64, np.array([[3, 4], [5, 6], [7, 8]], np.float32), np.ones(3, np.float32),
                      np.zeros((3, 128), np.uint8), np.zeros(3, np.int32))
    with gm.Context(device=0) as ctx:
        ctx.put_images({0: im, 1: im})
        labels = np.array([0, 1, 2, 0, 4, 5], np.int64)
        X, roots, nv = ctx.triangulate([0, 1], np.array([P, P]), labels)
        assert roots.tolist() == [0] and nv.tolist() == [2] and np.isnan(X).all()
        want = otri.triangulate([P, P], [im.xy[0], im.xy[0]])
        assert np.isnan(want).all()
        X, roots, nv = ctx.triangulate([0, 1], np.array([P, P]), np.arange(6, dtype=np.int64))
        assert roots.size == 0


def test_cap_and_errors(gm):
    sc = scenes.facade(n_images=6, n_kp=800, n_points=4000, n_pairs=10, min_covis=20)
    with gm.Context(device=0) as ctx:
        labels, Ps = _scene_tracks(gm, ctx, sc)
        ids = np.arange(6, dtype=np.int32)
        P = np.array(Ps).reshape(-1, 12)
        X, roots, nv = ctx.triangulate(ids, P, labels)
        T = roots.size
        assert T > 10
        Xs = np.full((T - 1, 3), 7.0)
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_triangulate(ctx.h, ids, P, labels, Xs, np.zeros(T - 1, np.int64), np.zeros(T - 1, np.int32), T - 1)
        assert e.value.status == gm.GM_ERR_NOMEM and e.value.required == T
        assert (Xs == 7.0).all()
        for bad_ids, bad_labels, status in [
            (ids[:5], labels, gm.GM_ERR_INVALID),                            # n_nodes differs from the images
            (np.array([0, 1, 2, 3, 4, 99], np.int32), labels, gm.GM_ERR_NOT_FOUND),
            (ids, np.where(np.arange(labels.size) == 3, 10, labels), gm.GM_ERR_INVALID),   # label above its node
        ]:
            with pytest.raises(gm.GeomatchError) as e:
                gm.gm_triangulate(ctx.h, bad_ids, P, bad_labels, np.empty((T, 3)), np.empty(T, np.int64),
                                  np.empty(T, np.int32), T)
            assert e.value.status == status
        v = int(np.nonzero(labels < np.arange(labels.size))[0][0])   # a node that is not its component's root
        lab2 = labels.copy()
        lab2[-1] = v                                                     # a label naming a non-root
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_triangulate(ctx.h, ids, P, lab2, np.empty((T, 3)), np.empty(T, np.int64), np.empty(T, np.int32), T)
        assert e.value.status == gm.GM_ERR_INVALID
        # outputs of mixed kinds (device X, host roots and n_views) are refused before any kernel runs
        import torch
        Xd = torch.full((T, 3), 7.0, dtype=torch.float64, device="cuda:0")
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_triangulate(ctx.h, ids, P, labels, Xd, np.empty(T, np.int64), np.empty(T, np.int32), T)
        assert e.value.status == gm.GM_ERR_INVALID and bool((Xd == 7.0).all())


# ---- per-image tracks (Sec. 6.3: each query image's features with their matches in all its candidate images)

def _image_track_obs(images, pairs, off, m):
    """Observations (image, feature) of every per-image track, in the track's order (own, then pairs in order)."""
    base = np.concatenate([[0], np.cumsum([im.n for im in images])]).astype(np.int64)
    obs = {}
    for k, p in enumerate(pairs):
        for i, j in m[off[k]:off[k + 1]]:
            v = int(base[p.a] + i)
            obs.setdefault(v, [(p.a, int(i))]).append((p.b, int(j)))
    return obs


def _check_image_tracks(images, Ps, pairs, off, m, X, nodes, nv, only_images=None):
    """Nodes and view counts equal the oracle's; every point within the perturbation bound of its track.  With
    `only_images`, the oracle runs on the pairs whose query image is listed (a query image's tracks depend only on
    its own pairs) and the GPU's tracks of those images are compared."""
    base = np.concatenate([[0], np.cumsum([im.n for im in images])]).astype(np.int64)
    keep = [k for k, p in enumerate(pairs) if only_images is None or p.a in only_images]
    want_nodes, want_nv, want_X = otri.image_tracks(
        Ps, [im.xy for im in images], [(pairs[k].a, pairs[k].b) for k in keep],
        [m[off[k]:off[k + 1]] for k in keep])
    if only_images is not None:
        img = np.searchsorted(base, nodes, side="right") - 1
        sel = np.isin(img, list(only_images))
        X, nodes, nv = X[sel], nodes[sel], nv[sel]
    np.testing.assert_array_equal(nodes, want_nodes)
    np.testing.assert_array_equal(nv, want_nv)
    obs = _image_track_obs(images, [pairs[k] for k in keep], np.concatenate([[0], np.cumsum(
        [off[k + 1] - off[k] for k in keep])]), np.concatenate([m[off[k]:off[k + 1]] for k in keep]))
    for t, v in enumerate(nodes):
        o = obs[int(v)]
        Pl, xy = [Ps[a] for a, _ in o], [images[a].xy[f] for a, f in o]
        if not np.isfinite(want_X[t]).all():
            assert np.isnan(X[t]).all()
            continue
        assert np.linalg.norm(X[t] - want_X[t]) <= _bound(Pl, xy, want_X[t]), (t, X[t], want_X[t])


def _pairs_with_reverse(sc, n):
    """The scene's first n pairs and the reverse of every other one (pairs in both directions, as Sec. 6.3
    describes: such feature pairs are triangulated once per image)."""
    pairs = list(sc.pairs[:n])
    pairs += [scenes.Pair(p.b, p.a, np.asarray(p.F, np.float32).reshape(3, 3).T.reshape(9).copy(), p.d, p.p, p.q)
              for p in sc.pairs[:n:2]]
    return pairs


def test_image_tracks_small_facade(gm):
    sc = scenes.facade(n_images=12, n_kp=1500, n_points=8000, n_pairs=40, min_covis=20)
    pairs = _pairs_with_reverse(sc, 40)
    Ps = [otri.camera_matrix(c) for c in sc.cameras]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m = ctx.match_pairs(pairs)
        ab = np.array([[p.a, p.b] for p in pairs], np.int32)
        X, nodes, nv = ctx.triangulate_image_tracks(list(range(12)), np.array(Ps), ab, off, m)
        X2, nodes2, nv2 = ctx.triangulate_image_tracks(list(range(12)), np.array(Ps), ab, off, m)
    assert nodes.size > 500 and nv.max() >= 3
    _check_image_tracks(sc.images, Ps, pairs, off, m, X, nodes, nv)
    # deterministic: every point's sums run in its track's order
    np.testing.assert_array_equal(X2, X)
    np.testing.assert_array_equal(nodes2, nodes)


def test_image_tracks_facade_device_buffers(gm, facade_scene):
    """The full facade batch (1200 pairs) with device matches, P and outputs; the tracks of five query images
    against the oracle."""
    import torch
    sc = facade_scene
    Ps = [otri.camera_matrix(c) for c in sc.cameras]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m = ctx.match_pairs(sc.pairs, device_out=True)
        cap = int(m.shape[0])
        X = torch.empty((cap, 3), dtype=torch.float64, device="cuda:0")
        nodes = torch.empty(cap, dtype=torch.int64, device="cuda:0")
        nv = torch.empty(cap, dtype=torch.int32, device="cuda:0")
        ab = np.array([[p.a, p.b] for p in sc.pairs], np.int32)
        n = gm.gm_triangulate_image_tracks(ctx.h, np.arange(len(sc.images), dtype=np.int32),
                                           torch.from_numpy(np.array(Ps).reshape(-1, 12)).cuda(), ab, off,
                                           m.contiguous(), X, nodes, nv, cap)
        X, nodes, nv = X[:n].cpu().numpy(), nodes[:n].cpu().numpy(), nv[:n].cpu().numpy()
        off, m = off.cpu().numpy(), m.cpu().numpy()
    assert n > 100000
    queries = {p.a for p in sc.pairs}
    pick = set(np.random.default_rng(3).choice(sorted(queries), 5, replace=False).tolist())
    _check_image_tracks(sc.images, Ps, sc.pairs, off, m, X, nodes, nv, only_images=pick)


def test_image_tracks_noise_free(gm):
    """True correspondences of exact projections as the matches of every ordered pair: each per-image track comes
    back at its point, with one view per image that sees it."""
    rng = np.random.default_rng(12)
    K = scenes.intrinsics(1000.0, 1280, 960)
    cams = []
    for k in range(5):
        c = np.array([2.0 * k - 4.0, 0.3 * k, -12.0])
        cams.append(scenes.camera_at(K, scenes.look_at(c, [0.0, 0.0, 0.0]), c))
    Xw = rng.uniform([-3, -2, -3], [3, 2, 3], (300, 3))
    images, pids = [], []
    for cam in cams:
        uv, z = scenes.project(cam, Xw)
        ok = rng.permutation(np.nonzero(scenes.inside(uv, 1280, 960) & (z > 0))[0])
        images.append(scenes.Image(1280, 960, uv[ok].astype(np.float32), np.ones(ok.size, np.float32),
                                   np.zeros((ok.size, 128), np.uint8), ok.astype(np.int32)))
        pids.append(ok)
    pairs, rows = [], []
    for a in range(5):
        for b in range(5):
            if a != b:
                where = {int(p): j for j, p in enumerate(pids[b])}
                rows.append(np.array([[i, where[int(p)]] for i, p in enumerate(pids[a]) if int(p) in where],
                                     np.int32).reshape(-1, 2))
                pairs.append(scenes.Pair(a, b, np.zeros(9, np.float32)))
    off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    m = np.concatenate(rows)
    Ps = [otri.camera_matrix(c) for c in cams]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(images)})
        X, nodes, nv = ctx.triangulate_image_tracks(list(range(5)), np.array(Ps),
                                                    np.array([[p.a, p.b] for p in pairs]), off, m)
    _check_image_tracks(images, Ps, pairs, off, m, X, nodes, nv)
    base = np.concatenate([[0], np.cumsum([im.n for im in images])])
    img = np.searchsorted(base, nodes, side="right") - 1
    pid = np.array([pids[k][v - base[k]] for k, v in zip(img, nodes)])
    seen = np.zeros(len(Xw), int)
    for p in pids:
        seen[p] += 1
    np.testing.assert_array_equal(nv, seen[pid])
    assert np.abs(X - Xw[pid]).max() < 2e-3



def test_image_tracks_many_views(gm):
    """Tracks of up to 70 views: query image 0 paired with 69 images and image 1 with 29, each true correspondence
    kept with a per-point probability, so one block of tracks mixes match counts from a few to 69 (past the solve
    pass's last count bin).  Every track against the oracle, and noise-free recovery."""
    rng = np.random.default_rng(70)
    K = scenes.intrinsics(1000.0, 1280, 960)
    cams = []
    for k in range(70):
        th = -1.0 + 2.0 * k / 69
        c = np.array([15.0 * np.sin(th), 0.5 * np.sin(3 * th), -15.0 * np.cos(th)])
        cams.append(scenes.camera_at(K, scenes.look_at(c, [0.0, 0.0, 0.0]), c))
    Xw = rng.uniform(-2.0, 2.0, (60, 3))
    keep_p = rng.uniform(0.05, 1.0, len(Xw))
    images = []
    for cam in cams:
        uv, z = scenes.project(cam, Xw)
        assert scenes.inside(uv, 1280, 960).all() and (z > 0).all()
        images.append(scenes.Image(1280, 960, uv.astype(np.float32), np.ones(len(Xw), np.float32),
                                   np.zeros((len(Xw), 128), np.uint8), np.arange(len(Xw), dtype=np.int32)))
    pairs, rows = [], []
    for a, bs in ((0, range(1, 70)), (1, range(2, 31))):
        for b in bs:
            keep = np.nonzero(rng.uniform(size=len(Xw)) < keep_p)[0]
            rows.append(np.stack([keep, keep], 1).astype(np.int32))
            pairs.append(scenes.Pair(a, b, np.zeros(9, np.float32)))
    off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    m = np.concatenate(rows)
    Ps = [otri.camera_matrix(c) for c in cams]
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(images)})
        X, nodes, nv = ctx.triangulate_image_tracks(list(range(70)), np.array(Ps),
                                                    np.array([[p.a, p.b] for p in pairs]), off, m)
    assert nv.max() >= 65 and nv.min() <= 10
    _check_image_tracks(images, Ps, pairs, off, m, X, nodes, nv)
    base = np.concatenate([[0], np.cumsum([im.n for im in images])])
    img = np.searchsorted(base, nodes, side="right") - 1
    assert np.abs(X - Xw[nodes - base[img]]).max() < 1e-4

def test_image_tracks_errors(gm):
    sc = scenes.facade(n_images=6, n_kp=800, n_points=4000, n_pairs=10, min_covis=20)
    Ps = np.array([otri.camera_matrix(c) for c in sc.cameras]).reshape(-1, 12)
    ids = np.arange(6, dtype=np.int32)
    with gm.Context(device=0) as ctx:
        ctx.put_images({k: im for k, im in enumerate(sc.images)})
        off, m = ctx.match_pairs(sc.pairs)
        ab = np.array([[p.a, p.b] for p in sc.pairs], np.int32)
        X, nodes, nv = ctx.triangulate_image_tracks(ids, Ps, ab, off, m)
        T = nodes.size
        assert T > 10
        Xs = np.full((T - 1, 3), 7.0)
        with pytest.raises(gm.GeomatchError) as e:
            gm.gm_triangulate_image_tracks(ctx.h, ids, Ps, ab, off, m, Xs, np.zeros(T - 1, np.int64),
                                           np.zeros(T - 1, np.int32), T - 1)
        assert e.value.status == gm.GM_ERR_NOMEM and e.value.required == T and (Xs == 7.0).all()
        k0 = int(np.nonzero(np.diff(off) >= 2)[0][0])   # a pair with two rows or more
        unsorted = m.copy()
        unsorted[off[k0]], unsorted[off[k0] + 1] = m[off[k0] + 1].copy(), m[off[k0]].copy()
        outside = m.copy()
        outside[off[k0], 1] = sc.images[sc.pairs[k0].b].n
        bad_off = off.copy()
        bad_off[0] = 1
        cases = [
            (ids, np.concatenate([ab, ab[:1]]), np.concatenate([off, off[-1:]]), m, gm.GM_ERR_INVALID),   # twice
            (ids, np.stack([ab[:, 0], ab[:, 0]], 1), off, m, gm.GM_ERR_INVALID),   # an image with itself
            (ids, ab, off, unsorted, gm.GM_ERR_INVALID),
            (ids, ab, off, outside, gm.GM_ERR_INVALID),
            (ids, ab, bad_off, m, gm.GM_ERR_INVALID),
            (ids[:5], ab, off, m, gm.GM_ERR_INVALID if ab.max() == 5 else gm.GM_OK),    # an image outside the list
            (np.array([0, 1, 2, 3, 4, 99], np.int32), ab, off, m, gm.GM_ERR_NOT_FOUND),
        ]
        for bad_ids, bad_ab, bad_o, bad_m, status in cases:
            if status == gm.GM_OK:
                continue
            with pytest.raises(gm.GeomatchError) as e:
                gm.gm_triangulate_image_tracks(ctx.h, bad_ids, Ps[:12 * len(bad_ids)] if len(bad_ids) < 6 else Ps,
                                               bad_ab, bad_o, bad_m, np.empty((T, 3)), np.empty(T, np.int64),
                                               np.empty(T, np.int32), T)
            assert e.value.status == status
        # no pairs, no tracks
        assert gm.gm_triangulate_image_tracks(ctx.h, ids, Ps, np.zeros((0, 2), np.int32), np.zeros(1, np.int64),
                                              np.zeros((0, 2), np.int32), np.empty((1, 3)), np.empty(1, np.int64),
                                              np.empty(1, np.int32), 1) == 0
