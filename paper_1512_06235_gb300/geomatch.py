"""ctypes binding of libgeomatch (include/geomatch.h): geometry-aware pairwise feature matching on a GB300.

Argument marshalling only -- every step of the matching runs in the CUDA library.  The functions ``gm_*`` mirror
the C entry points one to one; ``Context`` bundles them for convenience.  Device buffers may be torch CUDA
tensors (torch provides device memory and streams), host buffers numpy arrays.

The library must have been built (``python -m paper_1512_06235_gb300.build``); loading fails loudly otherwise.
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeomatch.so")

GM_OK, GM_ERR_INVALID, GM_ERR_NOMEM, GM_ERR_BUDGET, GM_ERR_NOT_FOUND, GM_ERR_CUDA, GM_ERR_TIMEOUT, \
    GM_ERR_CANCELLED, GM_ERR_BUSY = 0, -1, -2, -3, -4, -5, -6, -7, -8
GM_PATH_AUTO, GM_PATH_TC, GM_PATH_MMA, GM_PATH_SIMT = 0, 1, 2, 3
GM_OPT_PATH, GM_OPT_SCHEDULE, GM_OPT_CELL_PX, GM_OPT_GRAPH, GM_OPT_MMA_GROUP, GM_OPT_STREAM_CAP, GM_OPT_EVICT_LRU, \
    GM_OPT_TC_PIPE = 1, 2, 3, 4, 5, 6, 7, 8

_STATUS_NAMES = {0: "GM_OK", -1: "GM_ERR_INVALID", -2: "GM_ERR_NOMEM", -3: "GM_ERR_BUDGET", -4: "GM_ERR_NOT_FOUND",
                 -5: "GM_ERR_CUDA", -6: "GM_ERR_TIMEOUT", -7: "GM_ERR_CANCELLED", -8: "GM_ERR_BUSY"}

c_i32, c_i64, c_u16, c_u64, c_f32, c_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint16, ctypes.c_uint64, \
    ctypes.c_float, ctypes.c_void_p


class GmConfig(ctypes.Structure):
    _fields_ = [("device", c_i32), ("mem_budget_bytes", c_u64), ("max_inflight", c_i32), ("cuda_stream", c_p),
                ("path", c_i32), ("cell_px", c_i32), ("tuner_cache", ctypes.c_char_p)]


class GmPair(ctypes.Structure):
    _fields_ = [("img_a", c_i32), ("img_b", c_i32), ("F", c_f32 * 9), ("band_px", c_f32), ("ratio_num", c_u16),
                ("ratio_den", c_u16)]


class GmStats(ctypes.Structure):
    _fields_ = [("n_pairs", c_i64), ("n_queries", c_i64), ("n_candidates", c_i64), ("n_examined", c_i64),
                ("n_redecided", c_i64), ("n_matches", c_i64), ("ms_device", c_f32), ("ms_match", c_f32),
                ("path_used", c_i32), ("kernel_launches", c_i32), ("n_device_errors", c_i64),
                ("n_stream_reruns", c_i64), ("n_unstaged_groups", c_i64), ("cta_finish_spread", c_f32),
                ("reserved0", c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GmServingStats(ctypes.Structure):
    _fields_ = [("submitted", c_i64), ("completed", c_i64), ("failed", c_i64), ("batches", c_i64),
                ("max_batch_pairs", c_i64), ("peak_inflight_batches", c_i64), ("rejected_budget", c_i64),
                ("rejected_busy", c_i64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GmImage(ctypes.Structure):
    _fields_ = [("image_id", c_i32), ("width", c_i32), ("height", c_i32), ("n", c_i32), ("xy", c_p), ("scale", c_p),
                ("desc", c_p)]


class GmCoarseOpts(ctypes.Structure):
    _fields_ = [("eta_pct", c_i32), ("first_pct", c_i32), ("min_features", c_i32), ("min_matches", c_i32)]


class GmApproxStats(ctypes.Structure):
    _fields_ = [("n_groups", c_i64), ("n_candidates", c_i64), ("n_cells", c_i64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GmTuneResult(ctypes.Structure):
    _fields_ = [("path", c_i32), ("mma_group", c_i32), ("cell_px", c_i32), ("ms", ctypes.c_float),
                ("from_cache", c_i32), ("tc_pipe", c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GeomatchError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None

# C entry points: name -> (restype, argtypes)
_SIGNATURES = {
    "gm_create": (c_i32, [ctypes.POINTER(GmConfig), ctypes.POINTER(c_p)]),
    "gm_destroy": (c_i32, [c_p]),
    "gm_set_option": (c_i32, [c_p, c_i32, c_i64]),
    "gm_image_put": (c_i32, [c_p, c_i32, c_i32, c_i32, c_i32, c_p, c_p, c_p, c_i32]),
    "gm_image_evict": (c_i32, [c_p, c_i32]),
    "gm_image_info": (c_i32, [c_p, c_i32, ctypes.POINTER(c_i32)]),
    "gm_image_pin": (c_i32, [c_p, c_i32, c_i32]),
    "gm_selftest_wait": (c_i32, [c_p, c_i32, c_i32]),
    "gm_image_cache_stats": (c_i32, [c_p, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), ctypes.POINTER(c_i64),
                                     ctypes.POINTER(c_i64)]),
    "gm_match_pairs": (c_i32, [c_p, c_i32, ctypes.POINTER(GmPair), c_p, c_p, c_i64, ctypes.POINTER(c_i64)]),
    "gm_band_candidates": (c_i32, [c_p, ctypes.POINTER(GmPair), c_i32, c_i32, c_p, c_p, c_i64,
                                   ctypes.POINTER(c_i64)]),
    "gm_band_candidates_static": (c_i32, [c_p, ctypes.POINTER(GmPair), c_i32, c_i32, c_p, c_p, c_i64,
                                          ctypes.POINTER(c_i64)]),
    "gm_images_put": (c_i32, [c_p, c_i32, ctypes.POINTER(GmImage), c_i32]),
    "gm_merge_tracks": (c_i32, [c_p, c_i64, c_i64, c_p, c_p, ctypes.POINTER(c_i64)]),
    "gm_match_pairs_approx": (c_i32, [c_p, c_i32, ctypes.POINTER(GmPair), ctypes.c_float, c_p, c_p, c_i64,
                                      ctypes.POINTER(c_i64), ctypes.POINTER(GmApproxStats)]),
    "gm_coarse_prepare": (c_i32, [c_p, c_i32, c_p, ctypes.POINTER(GmCoarseOpts)]),
    "gm_coarse_selection": (c_i32, [c_p, c_i32, ctypes.POINTER(GmCoarseOpts), c_p, c_p, c_p, c_i32, c_p]),
    "gm_match_coarse": (c_i32, [c_p, c_i32, ctypes.POINTER(GmPair), ctypes.POINTER(GmCoarseOpts), c_p, c_p, c_i64,
                                ctypes.POINTER(c_i64), c_p]),
    "gm_triangulate": (c_i32, [c_p, c_i32, c_p, c_p, c_i64, c_p, c_i64, c_p, c_p, c_p, ctypes.POINTER(c_i64)]),
    "gm_triangulate_image_tracks": (c_i32, [c_p, c_i32, c_p, c_p, c_i32, c_p, c_p, c_p, c_i64, c_p, c_p, c_p,
                                            ctypes.POINTER(c_i64)]),
    "gm_select_pairs": (c_i32, [c_p, c_i32, c_i64, c_p, c_p, c_i32, c_i32, c_p, c_i64, ctypes.POINTER(c_i64)]),
    "gm_autotune": (c_i32, [c_p, c_i32, ctypes.POINTER(GmPair), c_i32, ctypes.POINTER(GmTuneResult)]),
    "gm_get_stats": (c_i32, [c_p, ctypes.POINTER(GmStats)]),
    "gm_submit": (c_i32, [c_p, ctypes.POINTER(GmPair), ctypes.POINTER(c_u64)]),
    "gm_poll": (c_i32, [c_p, c_u64, c_p, c_i64, ctypes.POINTER(c_i64), c_i32, ctypes.POINTER(ctypes.c_double)]),
    "gm_get_serving_stats": (c_i32, [c_p, ctypes.POINTER(GmServingStats)]),
    "gm_serving_drain": (c_i32, [c_p]),
    "gm_last_error": (ctypes.c_char_p, [c_p]),
}
EXPORTED = tuple(_SIGNATURES)


def load_library(path: str = LIB_PATH):
    """Loads libgeomatch.so (no fallback: raises if the CUDA library has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libgeomatch.so not found at {path}; build it with "
                          "`python -m paper_1512_06235_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, ctx=None):
    if status != GM_OK:
        msg = load_library().gm_last_error(ctx)
        raise GeomatchError(status, msg.decode() if msg else "")


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device, keepalive) of a numpy array or a torch tensor (contiguous)."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        x = x.contiguous()
        return x.data_ptr(), int(x.is_cuda), x
    a = np.ascontiguousarray(x)
    return a.ctypes.data, 0, a


def make_pair(a: int, b: int, F, d: float, p: int = 4, q: int = 5) -> GmPair:
    pr = GmPair()
    pr.img_a, pr.img_b = int(a), int(b)
    Fa = np.asarray(F, dtype=np.float32).reshape(9)
    for k in range(9):
        pr.F[k] = float(Fa[k])
    pr.band_px = float(d)
    pr.ratio_num, pr.ratio_den = int(p), int(q)
    return pr


_PAIR_DTYPE = np.dtype([("img_a", "<i4"), ("img_b", "<i4"), ("F", "<f4", (9,)), ("band_px", "<f4"),
                        ("ratio_num", "<u2"), ("ratio_den", "<u2")])


def make_pairs(a, b, F, d, p=4, q=5):
    """A ctypes array of gm_pair built from columns (vectorised; broadcast scalars): a, b int [n], F [n, 9] or
    [9], d, p, q.  Pass it to the C mirrors as the `pairs` argument to skip per-pair marshalling."""
    a = np.asarray(a)
    n = a.shape[0]
    rec = np.zeros(max(n, 1), _PAIR_DTYPE)
    rec["img_a"][:n] = a
    rec["img_b"][:n] = b
    rec["F"][:n] = np.broadcast_to(np.asarray(F, np.float32).reshape(-1, 9), (n, 9))
    rec["band_px"][:n] = d
    rec["ratio_num"][:n] = p
    rec["ratio_den"][:n] = q
    assert _PAIR_DTYPE.itemsize == ctypes.sizeof(GmPair)
    arr = (GmPair * max(n, 1)).from_buffer_copy(rec.tobytes())
    arr._n = n
    return arr


def _n_pairs(pairs):
    return getattr(pairs, "_n", len(pairs))


def _pairs_array(pairs):
    if isinstance(pairs, ctypes.Array):
        return pairs
    arr = (GmPair * max(1, len(pairs)))()
    for k, pr in enumerate(pairs):
        arr[k] = pr if isinstance(pr, GmPair) else make_pair(pr.a, pr.b, pr.F, pr.d, pr.p, pr.q)
    return arr


# ---------------------------------------------------------------------------------------------- C mirrors

def gm_create(device: int = 0, mem_budget_bytes: int = 0, max_inflight: int = 2, cuda_stream: int = 0,
              path: int = GM_PATH_AUTO, cell_px: int = 0, tuner_cache: str = None):
    lib = load_library()
    cfg = GmConfig(device, mem_budget_bytes, max_inflight, c_p(cuda_stream or None), path, cell_px,
                   tuner_cache.encode() if tuner_cache else None)
    h = c_p()
    _check(lib.gm_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def gm_destroy(ctx):
    _check(load_library().gm_destroy(ctx))


def gm_set_option(ctx, key: int, value: int):
    _check(load_library().gm_set_option(ctx, key, value), ctx)


def gm_image_put(ctx, image_id: int, width: int, height: int, xy, scale, desc):
    """xy float32 [n,2], scale float32 [n] (or None), desc uint8 [n,128]: numpy (host) or torch CUDA tensors."""
    n = int(xy.shape[0])
    pxy, dev_xy, k1 = _ptr(xy)
    psc, dev_sc, k2 = _ptr(scale)
    pds, dev_ds, k3 = _ptr(desc)
    if n and not (dev_xy == dev_ds and (scale is None or dev_sc == dev_xy)):
        raise ValueError("gm_image_put: xy, scale and desc must all be host or all be device memory")
    _check(load_library().gm_image_put(ctx, image_id, width, height, n, pxy, psc, pds, dev_xy), ctx)
    del k1, k2, k3


class ImageBatch:
    """A prebuilt gm_image array (the arrays' addresses, sizes and memory kind) for gm_images_put.  The arrays must
    stay alive and keep their addresses while the batch is used; their contents may change between calls."""

    def __init__(self, images):
        self.n = len(images)
        self.arr = (GmImage * max(1, self.n))()
        self.keep, devs = [], set()
        for k, (iid, w, h, xy, scale, desc) in enumerate(images):
            pxy, dxy, k1 = _ptr(xy)
            psc, dsc, k2 = _ptr(scale)
            pds, dds, k3 = _ptr(desc)
            self.keep += [k1, k2, k3]
            n = int(xy.shape[0])
            if n:
                devs.add(dxy)
                devs.add(dds)
                if scale is not None:
                    devs.add(dsc)
            self.arr[k] = GmImage(iid, w, h, n, pxy, psc, pds)
        if len(devs) > 1:
            raise ValueError("gm_images_put: all arrays must be host memory or all device memory")
        self.on_device = devs.pop() if devs else 0


def make_images(images) -> ImageBatch:
    """images: list of (image_id, width, height, xy, scale, desc), all host (numpy / pinned) or all device tensors."""
    return ImageBatch(images)


def gm_images_put(ctx, images):
    """images: an ImageBatch, or a list of (image_id, width, height, xy, scale, desc) (all host or all device)."""
    b = images if isinstance(images, ImageBatch) else ImageBatch(images)
    _check(load_library().gm_images_put(ctx, b.n, b.arr, b.on_device), ctx)


def gm_select_pairs(ctx, n_cams: int, point_off, point_cams, threshold: int, top_k: int, pairs, cap: int) -> int:
    """point_off int64 [P+1], point_cams int32, pairs int32 [cap, 3]: numpy or torch CUDA tensors."""
    po, _, k1 = _ptr(point_off)
    pc, _, k2 = _ptr(point_cams)
    pp, _, k3 = _ptr(pairs)
    n = c_i64(0)
    st = load_library().gm_select_pairs(ctx, n_cams, int(point_off.shape[0]) - 1, po, pc, threshold, top_k, pp, cap,
                                        ctypes.byref(n))
    if st == GM_ERR_NOMEM:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = n.value
        raise err
    _check(st, ctx)
    del k1, k2, k3
    return n.value


def gm_merge_tracks(ctx, n_nodes: int, edges, labels) -> int:
    """edges int64 [m, 2], labels int64 [n_nodes] (numpy or torch CUDA); returns the number of tracks."""
    pe, _, k1 = _ptr(edges)
    pl, _, k2 = _ptr(labels)
    nt = c_i64(0)
    _check(load_library().gm_merge_tracks(ctx, n_nodes, int(edges.shape[0]), pe, pl, ctypes.byref(nt)), ctx)
    del k1, k2
    return nt.value


def gm_triangulate(ctx, image_ids, P, labels, X, roots, n_views, cap: int) -> int:
    """image_ids int32 [K] (host), P float64 [K, 3, 4], labels int64 [n_nodes], X float64 [cap, 3], roots int64 [cap],
    n_views int32 [cap] (numpy or torch CUDA); returns the number of tracks (GeomatchError.required on NOMEM)."""
    ids = np.ascontiguousarray(image_ids, np.int32)
    pp, _, k1 = _ptr(P)
    pl, _, k2 = _ptr(labels)
    px, _, k3 = _ptr(X)
    pr, _, k4 = _ptr(roots)
    pv, _, k5 = _ptr(n_views)
    nt = c_i64(0)
    st = load_library().gm_triangulate(ctx, int(ids.shape[0]), ids.ctypes.data, pp, int(labels.shape[0]), pl, cap,
                                       px, pr, pv, ctypes.byref(nt))
    if st == GM_ERR_NOMEM and nt.value > cap:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = nt.value
        raise err
    _check(st, ctx)
    del k1, k2, k3, k4, k5
    return nt.value


def gm_triangulate_image_tracks(ctx, image_ids, P, pair_images, pair_off, matches, X, nodes, n_views, cap: int) -> int:
    """image_ids int32 [K] (host), P float64 [K, 3, 4], pair_images int32 [n_pairs, 2] (host), pair_off int64
    [n_pairs + 1] and matches int32 [M, 2] as gm_match_pairs wrote them, X float64 [cap, 3], nodes int64 [cap],
    n_views int32 [cap] (numpy or torch CUDA); returns the number of tracks (GeomatchError.required on NOMEM)."""
    ids = np.ascontiguousarray(image_ids, np.int32)
    ab = np.ascontiguousarray(pair_images, np.int32).reshape(-1, 2)
    pp, _, k1 = _ptr(P)
    po, _, k2 = _ptr(pair_off)
    pm, _, k3 = _ptr(matches)
    px, _, k4 = _ptr(X)
    pn, _, k5 = _ptr(nodes)
    pv, _, k6 = _ptr(n_views)
    nt = c_i64(0)
    st = load_library().gm_triangulate_image_tracks(ctx, int(ids.shape[0]), ids.ctypes.data, pp, int(ab.shape[0]),
                                                    ab.ctypes.data, po, pm, cap, px, pn, pv, ctypes.byref(nt))
    if st == GM_ERR_NOMEM and nt.value > cap:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = nt.value
        raise err
    _check(st, ctx)
    del k1, k2, k3, k4, k5, k6
    return nt.value


def coarse_opts(eta_pct: int = 20, first_pct: int = 10, min_features: int = 1000, min_matches: int = 4):
    return GmCoarseOpts(eta_pct, first_pct, min_features, min_matches)


def _coarse_pairs_array(pairs):
    if isinstance(pairs, ctypes.Array):
        return pairs
    if pairs and not any(isinstance(pr, GmPair) for pr in pairs):   # F and the band are not used
        return make_pairs([pr.a for pr in pairs], [pr.b for pr in pairs], np.eye(3), float("inf"),
                          [pr.p for pr in pairs], [pr.q for pr in pairs])
    arr = (GmPair * max(1, len(pairs)))()
    for k, pr in enumerate(pairs):
        arr[k] = pr if isinstance(pr, GmPair) else make_pair(pr.a, pr.b, np.eye(3), float("inf"), pr.p, pr.q)
    return arr


def gm_coarse_prepare(ctx, image_ids, opts=None):
    ids = np.ascontiguousarray(image_ids, np.int32)
    _check(load_library().gm_coarse_prepare(ctx, int(ids.size), ids.ctypes.data, opts), ctx)


def gm_coarse_selection(ctx, image_id: int, q1, q2, t, cap: int, opts=None):
    """Writes the selection lists into q1, q2, t (numpy or torch CUDA, cap entries each); returns the 3 sizes."""
    counts = np.zeros(3, np.int32)
    p1, _, k1 = _ptr(q1)
    p2, _, k2 = _ptr(q2)
    p3, _, k3 = _ptr(t)
    st = load_library().gm_coarse_selection(ctx, image_id, opts, p1, p2, p3, cap, counts.ctypes.data)
    if st == GM_ERR_NOMEM:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = int(counts.max())
        raise err
    _check(st, ctx)
    del k1, k2, k3
    return tuple(int(c) for c in counts)


def gm_match_coarse(ctx, pairs, pair_off, matches, cap: int, second=None, opts=None) -> int:
    """Coarse-stage matching into caller buffers (numpy or torch CUDA); returns n_written."""
    arr = _coarse_pairs_array(pairs)
    po, _, k1 = _ptr(pair_off)
    pm, _, k2 = _ptr(matches)
    ps, _, k3 = _ptr(second)
    n = c_i64(0)
    st = load_library().gm_match_coarse(ctx, _n_pairs(pairs), arr, opts, po, pm, cap, ctypes.byref(n), ps)
    if st == GM_ERR_NOMEM:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = n.value
        raise err
    _check(st, ctx)
    del k1, k2, k3
    return n.value


def gm_match_pairs_approx(ctx, pairs, pair_off, matches, cap: int, cell_scale: float = 1.0):
    """The paper's approximate matching into caller buffers (numpy or torch CUDA); returns (n_written, stats)."""
    arr = _pairs_array(pairs)
    po, _, k1 = _ptr(pair_off)
    pm, _, k2 = _ptr(matches)
    n = c_i64(0)
    stats = GmApproxStats()
    st = load_library().gm_match_pairs_approx(ctx, _n_pairs(pairs), arr, cell_scale, po, pm, cap, ctypes.byref(n),
                                              ctypes.byref(stats))
    if st == GM_ERR_NOMEM:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = n.value
        raise err
    _check(st, ctx)
    del k1, k2
    return n.value, stats.as_dict()


def gm_image_evict(ctx, image_id: int):
    _check(load_library().gm_image_evict(ctx, image_id), ctx)


def gm_image_info(ctx, image_id: int):
    """Keypoint count of a resident image, or None if it is not resident."""
    n = c_i32(0)
    st = load_library().gm_image_info(ctx, image_id, ctypes.byref(n))
    if st == GM_ERR_NOT_FOUND:
        return None
    _check(st, ctx)
    return n.value


def gm_selftest_wait(ctx, limit_us: int, set_flag: bool) -> int:
    """Status of the bounded device-wait self-test (GM_OK or GM_ERR_TIMEOUT); raises on other errors."""
    st = load_library().gm_selftest_wait(ctx, limit_us, 1 if set_flag else 0)
    if st not in (GM_OK, GM_ERR_TIMEOUT):
        _check(st, ctx)
    return st


def gm_image_pin(ctx, image_id: int, pin: bool = True):
    _check(load_library().gm_image_pin(ctx, image_id, 1 if pin else 0), ctx)


def gm_image_cache_stats(ctx) -> dict:
    a, b, w, c = c_i64(0), c_i64(0), c_i64(0), c_i64(0)
    _check(load_library().gm_image_cache_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(w),
                                               ctypes.byref(c)), ctx)
    return {"images": a.value, "bytes": b.value, "work_bytes": w.value, "evicted": c.value}


def gm_match_pairs(ctx, pairs, pair_off, matches, cap: int) -> int:
    """Low-level mirror: writes into caller buffers (numpy or torch CUDA); returns n_written.
    Raises GeomatchError (GM_ERR_NOMEM carries the required count in .required)."""
    arr = _pairs_array(pairs)
    po, _, k1 = _ptr(pair_off)
    pm, _, k2 = _ptr(matches)
    n = c_i64(0)
    st = load_library().gm_match_pairs(ctx, _n_pairs(pairs), arr, po, pm, cap, ctypes.byref(n))
    if st == GM_ERR_NOMEM:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = n.value
        raise err
    _check(st, ctx)
    del k1, k2
    return n.value


def gm_band_candidates(ctx, pair, query_begin: int, query_count: int, cand_off, cand, cap: int) -> int:
    arr = _pairs_array([pair])
    po, _, k1 = _ptr(cand_off)
    pc, _, k2 = _ptr(cand)
    n = c_i64(0)
    st = load_library().gm_band_candidates(ctx, arr, query_begin, query_count, po, pc, cap, ctypes.byref(n))
    if st == GM_ERR_NOMEM:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = n.value
        raise err
    _check(st, ctx)
    del k1, k2
    return n.value


def gm_band_candidates_static(ctx, pair, query_begin: int, query_count: int, cand_off, cand, cap: int) -> int:
    """gm_band_candidates with caller-owned device outputs and no allocation inside the call."""
    arr = _pairs_array([pair])
    po, _, k1 = _ptr(cand_off)
    pc, _, k2 = _ptr(cand)
    n = c_i64(0)
    st = load_library().gm_band_candidates_static(ctx, arr, query_begin, query_count, po, pc, cap, ctypes.byref(n))
    if st == GM_ERR_NOMEM:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = n.value
        raise err
    _check(st, ctx)
    del k1, k2
    return n.value


def gm_autotune(ctx, pairs, repeats: int = 3) -> dict:
    arr = _pairs_array(pairs)
    r = GmTuneResult()
    _check(load_library().gm_autotune(ctx, _n_pairs(pairs), arr, repeats, ctypes.byref(r)), ctx)
    return r.as_dict()


def gm_get_stats(ctx) -> dict:
    s = GmStats()
    _check(load_library().gm_get_stats(ctx, ctypes.byref(s)), ctx)
    return s.as_dict()


def gm_submit(ctx, pair) -> int:
    arr = _pairs_array([pair])
    t = c_u64(0)
    _check(load_library().gm_submit(ctx, arr, ctypes.byref(t)), ctx)
    return t.value


def gm_poll(ctx, ticket: int, matches: np.ndarray, timeout_ms: int = -1):
    """Returns (status, n, latency_us); status GM_OK or GM_ERR_TIMEOUT; other errors raise."""
    pm, _, keep = _ptr(matches)
    n = c_i64(0)
    lat = ctypes.c_double(0.0)
    st = load_library().gm_poll(ctx, ticket, pm, int(matches.shape[0]), ctypes.byref(n), timeout_ms,
                                ctypes.byref(lat))
    if st == GM_ERR_TIMEOUT:
        return st, 0, 0.0
    if st == GM_ERR_NOMEM:
        err = GeomatchError(st, load_library().gm_last_error(ctx).decode())
        err.required = n.value
        raise err
    _check(st, ctx)
    del keep
    return st, n.value, lat.value


def gm_get_serving_stats(ctx) -> dict:
    s = GmServingStats()
    _check(load_library().gm_get_serving_stats(ctx, ctypes.byref(s)), ctx)
    return s.as_dict()


def gm_serving_drain(ctx):
    _check(load_library().gm_serving_drain(ctx), ctx)


def gm_last_error(ctx=None) -> str:
    m = load_library().gm_last_error(ctx)
    return m.decode() if m else ""


# ---------------------------------------------------------------------------------------------- convenience

class Context:
    """A matcher context on one GPU: resident images, batch matching, candidate sets and serving."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_inflight: int = 2, stream=None,
                 path: int = GM_PATH_AUTO, cell_px: int = 0, tuner_cache: str = None):
        handle = 0
        if stream is not None:
            handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.h = gm_create(device, mem_budget_bytes, max_inflight, handle, path, cell_px, tuner_cache)
        self.n = {}
        self.device = device

    def close(self):
        if self.h:
            gm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key, value):
        gm_set_option(self.h, key, value)

    def put_image(self, image_id: int, image=None, *, width=None, height=None, xy=None, scale=None, desc=None):
        if image is not None:
            width, height, xy, scale, desc = image.width, image.height, image.xy, image.scale, image.desc
        gm_image_put(self.h, image_id, width, height, xy, scale, desc)
        self.n[image_id] = int(xy.shape[0])

    def put_images(self, images: dict):
        """images: {image_id: image} (objects with width, height, xy, scale, desc), registered in one call."""
        gm_images_put(self.h, [(k, im.width, im.height, im.xy, im.scale, im.desc) for k, im in images.items()])
        for k, im in images.items():
            self.n[k] = int(im.xy.shape[0])

    def evict(self, image_id: int):
        gm_image_evict(self.h, image_id)
        self.n.pop(image_id, None)

    def match_pairs(self, pairs, device_out: bool = False):
        """Returns (pair_off int64[P+1], matches int32[M,2]) as numpy arrays (or torch CUDA tensors)."""
        cap = sum(self.n.get(p.img_a if isinstance(p, GmPair) else p.a, 0) for p in pairs)
        if device_out:
            import torch
            off = torch.empty(len(pairs) + 1, dtype=torch.int64, device=f"cuda:{self.device}")
            m = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=f"cuda:{self.device}")
        else:
            off = np.empty(len(pairs) + 1, np.int64)
            m = np.empty((max(cap, 1), 2), np.int32)
        n = gm_match_pairs(self.h, pairs, off, m, cap)
        return off, m[:n]

    def band_candidates(self, pair, query_begin: int = 0, query_count=None):
        a = pair.img_a if isinstance(pair, GmPair) else pair.a
        b = pair.img_b if isinstance(pair, GmPair) else pair.b
        if query_count is None:
            query_count = self.n[a] - query_begin
        off = np.empty(query_count + 1, np.int64)
        cap = max(1, query_count * 64)
        while True:
            cand = np.empty(cap, np.int32)
            try:
                n = gm_band_candidates(self.h, pair, query_begin, query_count, off, cand, cap)
                return off, cand[:n]
            except GeomatchError as e:
                if e.status != GM_ERR_NOMEM:
                    raise
                cap = max(e.required, 1)
        del b

    def stats(self) -> dict:
        return gm_get_stats(self.h)

    def select_pairs(self, n_cams: int, point_off, point_cams, threshold: int = 8, top_k: int = 1 << 30):
        """Candidate pairs (Sec. 6.1) as int32 rows (a, b, count)."""
        cap = 1024
        while True:
            out = np.empty((cap, 3), np.int32)
            try:
                n = gm_select_pairs(self.h, n_cams, point_off, point_cams, threshold, top_k, out, cap)
                return out[:n]
            except GeomatchError as e:
                if e.status != GM_ERR_NOMEM:
                    raise
                cap = max(e.required, 1)

    def merge_tracks(self, n_nodes: int, edges):
        """(labels int64 [n_nodes], number of tracks) of the match graph."""
        labels = np.empty(n_nodes, np.int64)
        nt = gm_merge_tracks(self.h, n_nodes, np.ascontiguousarray(edges, np.int64).reshape(-1, 2), labels)
        return labels, nt

    def match_pairs_approx(self, pairs, cell_scale: float = 1.0):
        """Approximate matching (Sec. 6.2.1-6.2.2): (pair_off int64[P+1], matches int32[M,2], stats dict)."""
        cap = sum(self.n.get(p.img_a if isinstance(p, GmPair) else p.a, 0) for p in pairs)
        off = np.empty(_n_pairs(pairs) + 1, np.int64)
        m = np.empty((max(cap, 1), 2), np.int32)
        n, stats = gm_match_pairs_approx(self.h, pairs, off, m, cap, cell_scale)
        return off, m[:n], stats

    def coarse_selection(self, image_id: int, opts=None):
        """(q1, q2, t) ascending feature indices of the image's coarse selection (Sec. 4)."""
        cap = max(1, self.n.get(image_id, 1))
        q1, q2, t = (np.empty(cap, np.int32) for _ in range(3))
        c = gm_coarse_selection(self.h, image_id, q1, q2, t, cap, opts)
        return q1[:c[0]], q2[:c[1]], t[:c[2]]

    def match_coarse(self, pairs, opts=None):
        """Coarse-stage matching (Sec. 4): (pair_off int64[P+1], matches int32[M,2], second int32[P])."""
        cap = sum(self.n.get(p.img_a if isinstance(p, GmPair) else p.a, 0) for p in pairs)
        off = np.empty(len(pairs) + 1, np.int64)
        sec = np.empty(max(1, len(pairs)), np.int32)
        m = np.empty((max(cap, 1), 2), np.int32)
        n = gm_match_coarse(self.h, pairs, off, m, cap, sec, opts)
        return off, m[:n], sec[:len(pairs)]

    def triangulate(self, image_ids, P, labels):
        """Tracks of `labels` (image-major nodes over image_ids) as (X float64 [T, 3], roots int64 [T],
        n_views int32 [T]); P float64 [K, 3, 4]."""
        P = np.ascontiguousarray(P, np.float64).reshape(-1, 12)
        labels = np.ascontiguousarray(labels, np.int64)
        cap = 1024
        while True:
            X = np.empty((cap, 3), np.float64)
            roots = np.empty(cap, np.int64)
            nv = np.empty(cap, np.int32)
            try:
                n = gm_triangulate(self.h, image_ids, P, labels, X, roots, nv, cap)
                return X[:n], roots[:n], nv[:n]
            except GeomatchError as e:
                if e.status != GM_ERR_NOMEM or not hasattr(e, "required"):
                    raise
                cap = max(e.required, 1)

    def triangulate_image_tracks(self, image_ids, P, pair_images, pair_off, matches):
        """Per-image tracks of the matches of a gm_match_pairs call (pair_images [n_pairs, 2] image ids) as
        (X float64 [T, 3], nodes int64 [T], n_views int32 [T]); P float64 [K, 3, 4]."""
        P = np.ascontiguousarray(P, np.float64).reshape(-1, 12)
        cap = 1024
        while True:
            X = np.empty((cap, 3), np.float64)
            nodes = np.empty(cap, np.int64)
            nv = np.empty(cap, np.int32)
            try:
                n = gm_triangulate_image_tracks(self.h, image_ids, P, pair_images, pair_off, matches, X, nodes, nv,
                                                cap)
                return X[:n], nodes[:n], nv[:n]
            except GeomatchError as e:
                if e.status != GM_ERR_NOMEM or not hasattr(e, "required"):
                    raise
                cap = max(e.required, 1)

    def autotune(self, pairs, repeats: int = 3) -> dict:
        return gm_autotune(self.h, pairs, repeats)

    def submit(self, pair) -> int:
        return gm_submit(self.h, pair)

    def poll(self, ticket: int, timeout_ms: int = -1, cap: int = 1 << 16):
        """Returns (matches int32[M,2], latency_us), or None if the request is not done within timeout_ms."""
        while True:
            buf = np.empty((cap, 2), np.int32)
            try:
                st, n, lat = gm_poll(self.h, ticket, buf, timeout_ms)
            except GeomatchError as e:
                if e.status != GM_ERR_NOMEM:
                    raise
                cap = e.required
                continue
            if st == GM_ERR_TIMEOUT:
                return None
            return buf[:n], lat

    def serving_stats(self) -> dict:
        return gm_get_serving_stats(self.h)

    def serving_drain(self):
        gm_serving_drain(self.h)


def split_matches(pair_off, matches):
    """Per-pair list of (i, j) arrays from the CSR returned by match_pairs."""
    off = pair_off.cpu().numpy() if _is_torch(pair_off) else pair_off
    m = matches.cpu().numpy() if _is_torch(matches) else matches
    return [m[off[k]:off[k + 1]] for k in range(len(off) - 1)]


INF = math.inf
