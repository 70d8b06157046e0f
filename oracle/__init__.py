"""Plain FP64 CPU oracle for geometry-aware pairwise feature matching (arXiv 1512.06235, Sec. 6.2, App. A).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package; the product path (``paper_1512_06235_gb300``) never does.  The oracle shares no code
with the CUDA library.

The arithmetic lives in ``geomatch_oracle.c`` (compiled with ``-ffp-contract=off`` so that every FP64 step is a
separately rounded IEEE operation).  This module only builds it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geomatch_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so`` (if missing or older than its source)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.run(["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    f32p, u8p, i32p, i64p, f64p = (P(ctypes.c_float), P(ctypes.c_uint8), P(ctypes.c_int32),
                                  P(ctypes.c_int64), P(ctypes.c_double))
    lib.gmo_line.argtypes = [f32p, ctypes.c_float, ctypes.c_float, f64p]
    lib.gmo_line.restype = None
    lib.gmo_in_band.argtypes = [f64p, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    lib.gmo_in_band.restype = ctypes.c_int
    lib.gmo_dist2.argtypes = [u8p, u8p]
    lib.gmo_dist2.restype = ctypes.c_int32
    lib.gmo_band_set.argtypes = [f32p, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int32,
                                 f32p, i32p, ctypes.c_int64]
    lib.gmo_band_set.restype = ctypes.c_int64
    lib.gmo_match_pair.argtypes = [ctypes.c_int32, f32p, u8p, ctypes.c_int32, f32p, u8p, f32p, ctypes.c_float,
                                   ctypes.c_int32, ctypes.c_int32, i32p, i64p, i32p, i32p]
    lib.gmo_match_pair.restype = ctypes.c_int64
    lib.gmo_match_batch.argtypes = [ctypes.c_int32, i32p, P(f32p), P(u8p), ctypes.c_int32, i32p, f32p, f32p,
                                    i32p, i64p, i32p, i64p, ctypes.c_int32]
    lib.gmo_match_batch.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def line(F, x: float, y: float) -> np.ndarray:
    """Epipolar line l = F (x, y, 1)^T in FP64 (Sec. 6.2)."""
    lib = _load()
    Ff = _f32(np.asarray(F).reshape(9))
    out = np.zeros(3, np.float64)
    lib.gmo_line(_ptr(Ff, ctypes.c_float), float(x), float(y), _ptr(out, ctypes.c_double))
    return out


def in_band(l, d: float, x: float, y: float) -> bool:
    """Eqs. 2-3: |a x + b y + c| <= d * sqrt(a^2 + b^2), FP64, inclusive."""
    lib = _load()
    la = np.ascontiguousarray(l, dtype=np.float64)
    return bool(lib.gmo_in_band(_ptr(la, ctypes.c_double), float(d), float(x), float(y)))


def dist2(u, v) -> int:
    lib = _load()
    ua, va = _u8(u), _u8(v)
    return int(lib.gmo_dist2(_ptr(ua, ctypes.c_uint8), _ptr(va, ctypes.c_uint8)))


def band_set(F, d: float, xq: float, yq: float, xyB) -> np.ndarray:
    """Candidate set C_i (indices into B, ascending) of the query at (xq, yq): Eq. 2 by linear search."""
    lib = _load()
    Ff = _f32(np.asarray(F).reshape(9))
    xy = _f32(xyB).reshape(-1, 2)
    out = np.zeros(max(1, xy.shape[0]), np.int32)
    n = lib.gmo_band_set(_ptr(Ff, ctypes.c_float), float(d), float(xq), float(yq), xy.shape[0],
                         _ptr(xy, ctypes.c_float), _ptr(out, ctypes.c_int32), out.shape[0])
    return out[:n].copy()


def match_pair(xyA, descA, xyB, descB, F, d: float, p: int = 4, q: int = 5, with_dists: bool = False):
    """Match one pair.  Returns ``(match_j, n_cand)`` (or ``(match_j, n_cand, D1, D2)`` with ``with_dists``):
    ``match_j[i]`` is the index into B accepted for query i, or -1; ``n_cand`` is sum_i |C_i|."""
    lib = _load()
    xa, da, xb, db = _f32(xyA).reshape(-1, 2), _u8(descA).reshape(-1, 128), _f32(xyB).reshape(-1, 2), \
        _u8(descB).reshape(-1, 128)
    nA, nB = xa.shape[0], xb.shape[0]
    Ff = _f32(np.asarray(F).reshape(9))
    mj = np.full(max(1, nA), -1, np.int32)
    d1 = np.zeros(max(1, nA), np.int32)
    d2 = np.zeros(max(1, nA), np.int32)
    nc = np.zeros(1, np.int64)
    r = lib.gmo_match_pair(nA, _ptr(xa, ctypes.c_float), _ptr(da, ctypes.c_uint8), nB, _ptr(xb, ctypes.c_float),
                           _ptr(db, ctypes.c_uint8), _ptr(Ff, ctypes.c_float), float(d), int(p), int(q),
                           _ptr(mj, ctypes.c_int32), _ptr(nc, ctypes.c_int64), _ptr(d1, ctypes.c_int32),
                           _ptr(d2, ctypes.c_int32))
    if r < 0:
        raise ValueError("oracle: invalid arguments")
    if with_dists:
        return mj[:nA].copy(), int(nc[0]), d1[:nA].copy(), d2[:nA].copy()
    return mj[:nA].copy(), int(nc[0])


def match_batch(images, pairs, n_threads: int | None = None):
    """Match every pair on ``n_threads`` host threads.

    ``images``: sequence of objects with ``xy`` (float32[n,2]) and ``desc`` (uint8[n,128]).
    ``pairs``: sequence of objects with ``a``, ``b``, ``F`` (9 floats), ``d``, ``p``, ``q``.
    Returns ``(match_j_list, n_cand)``: per pair an int32[n_A] array (index into B or -1) and int64[n_pairs].
    """
    lib = _load()
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    xys = [_f32(im.xy).reshape(-1, 2) for im in images]
    dss = [_u8(im.desc).reshape(-1, 128) for im in images]
    img_n = np.array([x.shape[0] for x in xys], np.int32)
    f32p = ctypes.POINTER(ctypes.c_float)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    xy_arr = (f32p * max(1, len(xys)))(*[_ptr(x, ctypes.c_float) for x in xys])
    ds_arr = (u8p * max(1, len(dss)))(*[_ptr(x, ctypes.c_uint8) for x in dss])
    P = len(pairs)
    ab = np.array([[pr.a, pr.b] for pr in pairs], np.int32).reshape(-1, 2)
    Fs = np.array([np.asarray(pr.F, np.float32).reshape(9) for pr in pairs], np.float32).reshape(-1, 9)
    ds = np.array([pr.d for pr in pairs], np.float32)
    pq = np.array([[pr.p, pr.q] for pr in pairs], np.int32).reshape(-1, 2)
    nA = img_n[ab[:, 0]] if P else np.zeros(0, np.int32)
    off = np.zeros(max(1, P), np.int64)
    if P:
        off[1:P] = np.cumsum(nA.astype(np.int64))[:-1]
    total = int(nA.sum()) if P else 0
    mj = np.full(max(1, total), -1, np.int32)
    nc = np.zeros(max(1, P), np.int64)
    st = lib.gmo_match_batch(len(xys), _ptr(img_n, ctypes.c_int32), xy_arr, ds_arr, P,
                             _ptr(np.ascontiguousarray(ab), ctypes.c_int32), _ptr(np.ascontiguousarray(Fs),
                             ctypes.c_float), _ptr(ds, ctypes.c_float), _ptr(np.ascontiguousarray(pq), ctypes.c_int32),
                             _ptr(off, ctypes.c_int64), _ptr(mj, ctypes.c_int32), _ptr(nc, ctypes.c_int64),
                             int(n_threads))
    if st != 0:
        raise ValueError("oracle: invalid batch arguments")
    outs = [mj[off[k]:off[k] + nA[k]].copy() for k in range(P)]
    return outs, nc[:P].copy()


def matches_from_match_j(match_j: np.ndarray) -> np.ndarray:
    """(i, j) pairs sorted by i from a per-query match array (-1 = none)."""
    i = np.nonzero(match_j >= 0)[0].astype(np.int32)
    return np.stack([i, match_j[i].astype(np.int32)], axis=1) if i.size else np.zeros((0, 2), np.int32)
