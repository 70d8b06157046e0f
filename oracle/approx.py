"""Approximate geometry-aware matching as the paper describes it (arXiv 1512.06235, Sec. 6.2.1 grid-based search,
Sec. 6.2.2 dual-line grouping, App. A Steps 1-4) -- plain CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests and the CPU-baseline leg of ``bench.py`` may import this module; the product
path never does.  It shares no code with the CUDA library.

What it computes for a pair (A, B, F, d, p/q) with cell half-size h = d * cell_scale:

1. Grids (Sec. 6.2.1, Eqs. 6-9): four grids of 2h x 2h cells over B, offset by (0, 0), (h, 0), (0, h), (h, h).
   A point (x, y) lies in cell (i, j) = (floor((x - ox) / 2h), floor((y - oy) / 2h)) of the grid with offset
   (ox, oy); that cell's centre is (ox + (2i + 1) h, oy + (2j + 1) h).
2. Lines and groups (Sec. 6.2.2, App. A Step 2): every query's epipolar line l = F (x, y, 1) meets B's border
   [0, W] x [0, H] in a chord; its two ends, as positions t1 <= t2 along the border, are the query's key.  Queries
   sorted by (t1, t2, index) form groups: a query starts a new group when its t1 or t2 differs from those of the
   group's first query by more than 2 px.  Queries whose line misses the image each form their own group.
3. Candidates (Eqs. 4-5, App. A Step 3): on the chord of the group's first query, with K = ceil(|AB| / h), the
   K + 1 equidistant points x_k = (k x_A + (K - k) x_B) / K (k = 0 .. K); for each, the cell with the nearest centre
   among its four cells (ties: the lower grid); C' = every point of B binned into a chosen cell (a set).
4. Matching (App. A Step 4): for each query of the group, exact squared distances to C', nearest and second-nearest,
   the ratio test q^2 D1 < p^2 D2 with |C'| >= 2.

Readings (the paper is garbled or silent here):
- Eqs. 6-9 print centres as floor(x / 2d) d + 2d; the centres of 2d-cells offset by 0 or d are taken instead;
- K = ceil(|AB| / h) (the paper's |AB| / d is not an integer), the sample spacing is at most one cell half-size;
  a chord of length 0 gives the single point A;
- chord ends are ordered by the border position t (counter-clockwise from (0, 0): bottom edge t = x, right edge
  W + y, top edge 2W + H - x, left edge 2W + 2H - y; no wrap-around), A = the lower t;
- "within 2 pixels" compares t1 and t2 with the group's first query.  App. A Step 2's stencil compares with the
  previous query, but lines through a common epipole are nearly parallel, so in a dense query set consecutive
  lines are always closer than 2 px and that chain puts almost every query of a pair in one group; Sec. 6.2.2
  wants every query of a group to share one line;
- the geometry (lines, chords, keys, samples, cells) is FP32 with every operation rounded in the order written
  here (no fused multiply-add); the descriptor distances are exact integers;
- the group's candidate set comes from its first query's line; the 2-NN over C' is exact (no Kd-tree).
"""
from __future__ import annotations

import math

import numpy as np

f32 = np.float32


def line32(F, x, y):
    """(a, b, c) = F (x, y, 1) in FP32: ((F0 x + F1 y) + F2), each operation rounded."""
    F = np.asarray(F, np.float32).reshape(9)
    x, y = f32(x), f32(y)
    a = (F[0] * x + F[1] * y) + F[2]
    b = (F[3] * x + F[4] * y) + F[5]
    c = (F[6] * x + F[7] * y) + F[8]
    return f32(a), f32(b), f32(c)


def border_t(x, y, W, H):
    """Position of a border point along the border (counter-clockwise from the origin), FP32."""
    W, H = f32(W), f32(H)
    if y == 0:
        return f32(x)
    if x == W:
        return f32(W + y)
    if y == H:
        return f32(f32(W + H) + f32(W - x))
    return f32(f32(2 * W + H) + f32(H - y))


def chord(a, b, c, W, H):
    """((xA, yA, tA), (xB, yB, tB)) ends of the line inside [0, W] x [0, H] with tA <= tB, or None."""
    W, H = f32(W), f32(H)
    zero = f32(0.0)
    cand = []
    if b != 0:
        y0 = f32(-c / b)
        if zero <= y0 <= H:
            cand.append((zero, y0))
        yW = f32(-f32(a * W + c) / b)
        if zero <= yW <= H:
            cand.append((W, yW))
    if a != 0:
        x0 = f32(-c / a)
        if zero <= x0 <= W:
            cand.append((x0, zero))
        xH = f32(-f32(b * H + c) / a)
        if zero <= xH <= W:
            cand.append((xH, H))
    if not cand:
        return None
    ts = [border_t(x, y, W, H) for x, y in cand]
    lo = min(range(len(cand)), key=lambda k: (ts[k], k))
    hi = min(range(len(cand)), key=lambda k: (-ts[k], k))
    return (cand[lo][0], cand[lo][1], ts[lo]), (cand[hi][0], cand[hi][1], ts[hi])


def samples(ends, h):
    """The equidistant points of Eqs. 4-5 on the chord (FP32 arrays xs, ys)."""
    (xa, ya, _), (xb, yb, _) = ends
    h = f32(h)
    dx, dy = f32(xb - xa), f32(yb - ya)
    L = f32(np.sqrt(f32(f32(dx * dx) + f32(dy * dy))))
    K = int(math.ceil(float(f32(L / h))))
    if K == 0:
        return np.array([xa], np.float32), np.array([ya], np.float32)
    k = np.arange(K + 1, dtype=np.float32)
    Kf = f32(K)
    xs = ((k * xa).astype(np.float32) + ((Kf - k) * xb).astype(np.float32)).astype(np.float32) / Kf
    ys = ((k * ya).astype(np.float32) + ((Kf - k) * yb).astype(np.float32)).astype(np.float32) / Kf
    return xs.astype(np.float32), ys.astype(np.float32)


def cell_of(g, x, y, h):
    """(i, j) of the point in grid g (offset ((g & 1) h, (g >> 1) h)), FP32."""
    h = f32(h)
    h2 = f32(h + h)
    ox = h if g & 1 else f32(0.0)
    oy = h if g >> 1 else f32(0.0)
    i = np.floor(((np.asarray(x, np.float32) - ox).astype(np.float32) / h2).astype(np.float32)).astype(np.int64)
    j = np.floor(((np.asarray(y, np.float32) - oy).astype(np.float32) / h2).astype(np.float32)).astype(np.int64)
    return i, j


def chosen_cells(xs, ys, h):
    """For every sample the (grid, i, j) of the cell whose centre is nearest (ties: the lower grid)."""
    h = f32(h)
    best_d, best = None, None
    for g in range(4):
        ox = h if g & 1 else f32(0.0)
        oy = h if g >> 1 else f32(0.0)
        i, j = cell_of(g, xs, ys, h)
        cx = (ox + ((2 * i + 1).astype(np.float32) * h).astype(np.float32)).astype(np.float32)
        cy = (oy + ((2 * j + 1).astype(np.float32) * h).astype(np.float32)).astype(np.float32)
        dx = (xs - cx).astype(np.float32)
        dy = (ys - cy).astype(np.float32)
        d2 = ((dx * dx).astype(np.float32) + (dy * dy).astype(np.float32)).astype(np.float32)
        cur = np.stack([np.full(i.shape, g), i, j], 1)
        if best is None:
            best_d, best = d2, cur
        else:
            take = d2 < best_d
            best_d = np.where(take, d2, best_d)
            best[take] = cur[take]
    return best


def bins(xyB, h):
    """Grid binning of B's points (App. A Step 1): {(g, i, j): [point indices]}."""
    xyB = np.asarray(xyB, np.float32).reshape(-1, 2)
    out = {}
    for g in range(4):
        i, j = cell_of(g, xyB[:, 0], xyB[:, 1], h)
        for p in range(xyB.shape[0]):
            out.setdefault((g, int(i[p]), int(j[p])), []).append(p)
    return out


def groups(F, xyA, W, H):
    """Sorted query order and the groups as lists of query indices (App. A Step 2); plus every query's chord."""
    xyA = np.asarray(xyA, np.float32).reshape(-1, 2)
    keyed, lineless, ends = [], [], []
    two = f32(2.0)
    for q in range(xyA.shape[0]):
        a, b, c = line32(F, xyA[q, 0], xyA[q, 1])
        e = chord(a, b, c, W, H)
        ends.append(e)
        if e is None:
            lineless.append(q)
        else:
            keyed.append((float(e[0][2]), float(e[1][2]), q))
    keyed.sort()
    out = []
    lead = None
    for t1, t2, q in keyed:
        if lead is None or abs(f32(f32(t1) - f32(lead[0]))) > two or abs(f32(f32(t2) - f32(lead[1]))) > two:
            out.append([q])
            lead = (t1, t2)
        else:
            out[-1].append(q)
    out += [[q] for q in lineless]
    return out, ends


def candidate_set(ends, h, binned):
    """C' of a chord: ascending indices of B's points in the chosen cells."""
    if ends is None:
        return np.zeros(0, np.int64)
    xs, ys = samples(ends, h)
    members = set()
    for g, i, j in chosen_cells(xs, ys, h).tolist():
        members.update(binned.get((g, i, j), ()))
    return np.array(sorted(members), np.int64)


def match_pair(xyA, descA, xyB, descB, W, H, F, d, p=4, q=5, cell_scale=1.0, with_stats=False):
    """match_j[i] (index into B or -1) for every query of A; with_stats also (groups, sum over queries of |C'|)."""
    h = f32(f32(d) * f32(cell_scale))
    binned = bins(xyB, h)
    gs, ends = groups(F, xyA, W, H)
    dA = np.asarray(descA, np.int64).reshape(-1, 128)
    dB = np.asarray(descB, np.int64).reshape(-1, 128)
    mj = np.full(dA.shape[0], -1, np.int32)
    total = 0
    for grp in gs:
        C = candidate_set(ends[grp[0]], h, binned)
        total += C.size * len(grp)
        if C.size < 2:
            continue
        for qi in grp:
            D = ((dB[C] - dA[qi]) ** 2).sum(1)
            order = np.lexsort((C, D))
            D1, D2 = int(D[order[0]]), int(D[order[1]])
            if q * q * D1 < p * p * D2:
                mj[qi] = int(C[order[0]])
    if with_stats:
        return mj, len(gs), total
    return mj
