// gm_band.cuh -- epipolar band of one query and the exact cell walk over the resident grid of image B.
//
// Sec. 6.2, Eqs. 2-3: p' is a candidate of the query p iff |a x' + b y' + c| <= d sqrt(a^2 + b^2) with
// (a, b, c) = F (x, y, 1)^T.  The reference definition evaluates this in FP64 (left-to-right sums, no fused
// multiply-add).  Here every visited point is first tested in FP32 against two thresholds that bracket the FP64
// threshold by a proven bound on the FP32 error; only points between the two thresholds are re-decided with the
// FP64 expression, evaluated operation by operation in the same order, so the set is exactly the FP64 set.
//
// FP32 error bound (u = 2^-24; every quantity below is for the query's line and any point 0 <= x' < W,
// 0 <= y' < H):
//   a32 = fma(F0, x, fma(F1, y, F2)) differs from the FP64 value by at most 2.002 u (|F0 x| + |F1 y| + |F2|),
//   likewise b32, c32 (the FP64 value is within 2^-52 of the exact one);
//   s32 = fma(a32, x', fma(b32, y', c32)) differs from the FP64 s by at most
//       2.01 u (|a32| W + |b32| H + |c32|) + 2.002 u (A W + B H + C)         =: E_s
//   where A, B, C are the absolute sums of the three rows above;
//   d * sqrt(a32^2 + b32^2) differs from the FP64 threshold by at most d (4.02 u n + 2.002 u (A + B)) =: E_t.
// The code uses 2.5 u / 5 u factors, which also absorb the rounding of computing the bound itself.  A point with
// |s32| <= thr - E is inside, |s32| > thr + E is outside, anything between is re-decided in FP64.  Every point
// within 1e-4 px of the band edge is re-decided as well (E >= 1e-4 n).
#pragma once
#include <cmath>
#include <cstdint>

#include "gm_internal.h"

namespace gm {

enum BandMode : int { kBandNormal = 0, kBandAll = 1, kBandEmpty = 2, kBandSlow = 3 };

struct BandLine {
    float a, b, c;          // FP32 line
    float thr_lo, thr_hi;   // |s32| <= thr_lo: inside; |s32| > thr_hi: outside; else FP64 re-decision
    float t_walk;           // half-width (in |s| units) that the cell walk must cover
    int mode;
};

constexpr float kU = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of FP32

__device__ __forceinline__ BandLine band_line(const float F[9], float x, float y, float d, float W, float H)
{
    BandLine L;
    L.a = fmaf(F[0], x, fmaf(F[1], y, F[2]));
    L.b = fmaf(F[3], x, fmaf(F[4], y, F[5]));
    L.c = fmaf(F[6], x, fmaf(F[7], y, F[8]));
    L.thr_lo = L.thr_hi = L.t_walk = 0.0f;
    if (isinf(d)) { L.mode = kBandAll; return L; }
    const float ax = fabsf(x), ay = fabsf(y);
    const float Ar = fmaf(fabsf(F[0]), ax, fmaf(fabsf(F[1]), ay, fabsf(F[2])));
    const float Br = fmaf(fabsf(F[3]), ax, fmaf(fabsf(F[4]), ay, fabsf(F[5])));
    const float Cr = fmaf(fabsf(F[6]), ax, fmaf(fabsf(F[7]), ay, fabsf(F[8])));
    const float n = sqrtf(fmaf(L.a, L.a, L.b * L.b));
    const float M32 = fmaf(fabsf(L.a), W, fmaf(fabsf(L.b), H, fabsf(L.c)));
    const float MF = fmaf(Ar, W, fmaf(Br, H, Cr));
    const float Es = 2.5f * kU * (M32 + MF);
    const float thr = d * n;
    const float Et = d * (5.0f * kU * n + 2.5f * kU * (Ar + Br));
    float E = (Es + Et) * (1.0f + 16.0f * kU);
    E = fmaxf(E, 1.0001e-4f * n);
    L.thr_lo = thr - E;
    L.thr_hi = thr + E;
    L.t_walk = L.thr_hi + Es;
    const bool sane = n > 1e-30f && isfinite(L.t_walk) && isfinite(M32) && isfinite(MF) && M32 < 1e30f &&
                      MF < 1e30f;
    L.mode = sane ? kBandNormal : kBandSlow;
    return L;
}

// The reference decision of Eqs. 2-3 in FP64, operation by operation: a = (F0 x + F1 y) + F2 etc.,
// n = sqrt(a a + b b), inside iff |(a x' + b y') + c| <= d n; a == b == 0 gives no band.
__device__ __forceinline__ bool band_exact(const float F[9], float x, float y, float d, float xp, float yp)
{
    const double X = (double)x, Y = (double)y;
    const double a = __dadd_rn(__dadd_rn(__dmul_rn((double)F[0], X), __dmul_rn((double)F[1], Y)), (double)F[2]);
    const double b = __dadd_rn(__dadd_rn(__dmul_rn((double)F[3], X), __dmul_rn((double)F[4], Y)), (double)F[5]);
    const double c = __dadd_rn(__dadd_rn(__dmul_rn((double)F[6], X), __dmul_rn((double)F[7], Y)), (double)F[8]);
    const double n = __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)));
    if (n == 0.0) return false;
    const double thr = __dmul_rn((double)d, n);
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(a, (double)xp), __dmul_rn(b, (double)yp)), c);
    return fabs(s) <= thr;
}

// The same decision split in two: the FP64 line and threshold of a query (once), then the test of a point.  Every
// operation is the one band_exact performs, in the same order, so the outcome is identical; a == b == 0 gives the
// threshold -1 (no point is inside, as band_exact returns false).
struct BandLine64 {
    double a, b, c, thr;
};

__device__ __forceinline__ BandLine64 band_line64(const float F[9], float x, float y, float d)
{
    const double X = (double)x, Y = (double)y;
    BandLine64 L;
    L.a = __dadd_rn(__dadd_rn(__dmul_rn((double)F[0], X), __dmul_rn((double)F[1], Y)), (double)F[2]);
    L.b = __dadd_rn(__dadd_rn(__dmul_rn((double)F[3], X), __dmul_rn((double)F[4], Y)), (double)F[5]);
    L.c = __dadd_rn(__dadd_rn(__dmul_rn((double)F[6], X), __dmul_rn((double)F[7], Y)), (double)F[8]);
    const double n = __dsqrt_rn(__dadd_rn(__dmul_rn(L.a, L.a), __dmul_rn(L.b, L.b)));
    L.thr = n == 0.0 ? -1.0 : __dmul_rn((double)d, n);
    return L;
}

static __device__ __noinline__ bool band_test64_call(double a, double b, double c, double thr, float xp, float yp)
{
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(a, (double)xp), __dmul_rn(b, (double)yp)), c);
    return fabs(s) <= thr;
}

// Out-of-line copy of band_exact for unrolled epilogues: the rare FP64 re-decision stays one call instead of
// being inlined at every element (which would flood the instruction cache).
static __device__ __noinline__ bool band_exact_call(const float *F, float x, float y, float d, float xp, float yp)
{
    return band_exact(F, x, y, d, xp, yp);
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Cell range [c0, c1] of grid line k (a column for a column walk, a row otherwise) that the strip
// |pa u + pb v + c| <= T can touch for u in [k cs, (k+1) cs); returns false if none.
__device__ __forceinline__ bool strip_range(float pa, float pb, float c, float T, int k, float cs, float inv_cs,
                                            float ulim, float vlim, int ng, int &c0, int &c1)
{
    const float u0 = (float)k * cs;
    const float u1 = fminf(u0 + cs, ulim);
    const float ib = 1.0f / pb;
    const float v0 = -fmaf(pa, u0, c) * ib;
    const float v1 = -fmaf(pa, u1, c) * ib;
    const float h = T * fabsf(ib);
    const float pad = 8.0f * kU * (fabsf(pa) * ulim + fabsf(c) + T) * fabsf(ib) + 1e-3f;
    const float lo = fminf(v0, v1) - h - pad;
    const float hi = fmaxf(v0, v1) + h + pad;
    if (!(hi >= 0.0f) || !(lo < vlim)) return false;
    c0 = (int)floorf(fmaxf(lo, 0.0f) * inv_cs);
    c1 = (int)floorf(fminf(hi, vlim) * inv_cs);
    c1 = min(c1, ng - 1);
    c0 = max(c0, 0);
    return c0 <= c1;
}

// Warp-cooperative walk over every point of B that may lie in the band of the query (x, y).  For each chunk of
// up to 32 visited points it calls visit(valid, inside, colpos) on all 32 lanes (a warp-uniform call); colpos is
// the column-major position of the lane's point.  Counters are per lane (sum them over the warp).
template <class Visit>
__device__ __forceinline__ void band_walk(const ImageDev &B, const BandLine &L, const float F[9], float qx, float qy,
                                          float d, Visit &&visit, unsigned &examined, unsigned &redecided)
{
    const int lane = threadIdx.x & 31;
    if (L.mode == kBandEmpty) return;
    if (L.mode == kBandAll || L.mode == kBandSlow) {
        for (int base = 0; base < B.n; base += 32) {
            const int pos = base + lane;
            const bool valid = pos < B.n;
            bool inb = valid;
            if (valid && L.mode == kBandSlow) {
                const float2 p = B.xy[pos];
                inb = band_exact(F, qx, qy, d, p.x, p.y);
                ++redecided;
            }
            examined += valid;
            visit(valid, inb, pos);
        }
        return;
    }
    const bool colwise = fabsf(L.b) >= fabsf(L.a);
    const float cs = (float)(1 << B.cell_shift), inv_cs = 1.0f / cs;
    const float W = (float)B.width, H = (float)B.height;
    const int nlines = colwise ? B.gx : B.gy;
    const int ng = colwise ? B.gy : B.gx;
    const float pa = colwise ? L.a : L.b, pb = colwise ? L.b : L.a;
    const float ulim = colwise ? W : H, vlim = colwise ? H : W;
    const int32_t *offs = colwise ? B.col_off : B.row_off;
    const float2 *pts = colwise ? B.xy : B.xy_r;
    for (int base = 0; base < nlines; base += 32) {
        const int k = base + lane;
        int start = 0, len = 0, c0, c1;
        if (k < nlines && strip_range(pa, pb, L.c, L.t_walk, k, cs, inv_cs, ulim, vlim, ng, c0, c1)) {
            const int32_t *o = offs + (int64_t)k * ng;
            start = o[c0];
            len = o[c1 + 1] - start;
        }
        // inclusive scan of run lengths over the warp -> exclusive offsets
        int incl = len;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, s);
            if (lane >= s) incl += v;
        }
        const int excl = incl - len;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int p0 = 0; p0 < total; p0 += 32) {
            const int p = p0 + lane;
            // largest run r with excl[r] <= p (runs of length 0 are skipped automatically)
            int r = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int cand = r + step;
                const int v = __shfl_sync(0xffffffffu, excl, cand & 31);
                if (cand < 32 && v <= p) r = cand;
            }
            const int rs = __shfl_sync(0xffffffffu, start, r);
            const int re = __shfl_sync(0xffffffffu, excl, r);
            const bool valid = p < total;
            bool inb = false;
            int pos = 0;
            if (valid) {
                pos = rs + (p - re);
                const float2 pt = pts[pos];
                const float s = fmaf(L.a, pt.x, fmaf(L.b, pt.y, L.c));
                const float as = fabsf(s);
                inb = as <= L.thr_lo;
                if (!inb && as <= L.thr_hi) {
                    inb = band_exact(F, qx, qy, d, pt.x, pt.y);
                    ++redecided;
                }
                if (!colwise) pos = B.idx_r[pos];
                ++examined;
            }
            visit(valid, inb, pos);
        }
    }
}

}  // namespace gm
