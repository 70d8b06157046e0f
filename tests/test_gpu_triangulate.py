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
