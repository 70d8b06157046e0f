// gm_match_mma.cu -- tensor-core matching path: query groups x candidate chunks on mma.sync s8 (exact int32).
//
// App. A Steps 3-4 for a group of 16*MT consecutive queries of one pair (queries are sorted by the position of
// their epipolar line, so a group's bands nearly coincide; the paper groups lines within 2 px the same way, Sec.
// 6.2.2, but here every query still gets its own exact band):
//   1. each query's FP32 line and exact-decision thresholds (gm_band.cuh);
//   2. one walk over B's grid for the whole group: the union of the group's strips lies between two chords of
//      the strips' upper and lower envelopes (a maximum of linear functions is convex, so it lies below the chord
//      between its end values, and a minimum lies above its chord), so one run of cells per grid column covers
//      every point any query of the group can accept;
//   3. the candidate stream is cut into chunks of 64 keypoints; descriptors (recentred int8), coordinates and
//      norms are staged in shared memory with cp.async, double-buffered;
//   4. exact dot products a'.b' of the 16*MT x 64 tile by mma.sync.m16n8k32.s32.s8.s8 (K = 128 in 4 steps);
//   5. fused epilogue per element: the query's exact band test, D = |a'|^2 + |b'|^2 - 2 a'.b' packed with the
//      column into one int32 key (D * 256 + column; D < 2^23), masked running top-2 with three integer min/max,
//      and the candidate count;
//   6. a quad / cross-warp merge of the top-2 states and the integer ratio test q^2 D1 < p^2 D2.
// With p < q a tie D1 == D2 is rejected whatever the tie-break, so the packed column bits never decide a match.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "gm_band.cuh"
#include "gm_internal.h"

namespace gm {
namespace {

constexpr int kN = 64;             // candidates per chunk
constexpr int kStages = 4;         // chunks in flight per block (cp.async ring)
constexpr int kWarps = 4;          // warp w owns columns [16 w, 16 w + 16) of a chunk (two n8 tiles)
constexpr int kThreads = kWarps * 32;
constexpr int kMinBlocks = 4;      // blocks per SM the register budget is sized for
constexpr int kPitch = 144;        // shared bytes per descriptor row: 128 + 16 makes fragment loads conflict-free
constexpr int kMaxRuns = 512;      // grid lines per walk pass
constexpr int kCounterShards = 64;

template <int MT>
struct Smem {
    alignas(16) int8_t qdesc[16 * MT][kPitch];
    alignas(16) int8_t bdesc[kStages][kN][kPitch];
    alignas(16) float2 bxy[kStages][kN];
    alignas(16) int32_t bnb[kStages][kN];
    int32_t bpos[kStages][kN];
    float ln[16 * MT][8];          // a, b, c, thr_lo, thr_hi, qx, qy, -
    int32_t rinfo[16 * MT][4];     // A position, original index, |a'|^2 * 256, valid
    int32_t run_start[kMaxRuns];
    int32_t run_excl[kMaxRuns + 1];
    float env[4];                  // chord ends: top(0), top(ulim), bot(0), bot(ulim)
    int32_t red[kWarps][16 * MT][4];
    float F[9];
    int32_t walk_full, colwise;
    int64_t item;
    unsigned long long stat[3];
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void mma_s8(int (&d)[4], const int (&a)[4], int b0, int b1)
{
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct Top2Key {
    int k1, k2, j1, cnt;
};

__device__ __forceinline__ void merge_top2(Top2Key &t, int ok1, int ok2, int oj1, int ocnt)
{
    const int nk2 = min(max(t.k1, ok1), min(t.k2, ok2));
    if (ok1 < t.k1) { t.k1 = ok1; t.j1 = oj1; }
    t.k2 = nk2;
    t.cnt += ocnt;
}

__device__ __forceinline__ int pair_of_item(const int64_t *__restrict__ item_off, int n_pairs, int64_t t)
{
    int lo = 0, hi = n_pairs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (item_off[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int MT>
__global__ void __launch_bounds__(kThreads, kMinBlocks) match_mma_kernel(
    const ImageDev *__restrict__ imgs, const PairDev *__restrict__ pairs, const int64_t *__restrict__ item_off,
    int32_t n_pairs, const int32_t *__restrict__ qorder, int64_t item_begin, int64_t item_end, int32_t persistent,
    int32_t *__restrict__ next, int32_t *__restrict__ match_j, BatchCounters *__restrict__ ctr)
{
    constexpr int G = 16 * MT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<MT> &sm = *reinterpret_cast<Smem<MT> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    if (tid < 3) sm.stat[tid] = 0ull;
    unsigned long long my_cand = 0, my_exam = 0, my_redec = 0;

    for (int64_t it = 0;; ++it) {
        __syncthreads();
        if (tid == 0) {
            if (persistent) sm.item = item_begin + atomicAdd(next, 1);
            else sm.item = it == 0 ? item_begin + blockIdx.x : item_end;
        }
        __syncthreads();
        const int64_t item = sm.item;
        if (item >= item_end) break;
        const int pi = pair_of_item(item_off, n_pairs, item);
        const PairDev &P = pairs[pi];
        const ImageDev &A = imgs[P.a];
        const ImageDev &B = imgs[P.b];
        const int q0 = (int)(item - item_off[pi]) * G;
        const float d = P.d;
        const float W = (float)B.width, H = (float)B.height;

        // ---- 1. queries: lines, thresholds, descriptors
        if (tid < 9) sm.F[tid] = P.F[tid];
        __syncthreads();
        if (tid < G) {
            const int k = q0 + tid;
            float *L = sm.ln[tid];
            int32_t *ri = sm.rinfo[tid];
            if (k < P.n_a) {
                const int s = qorder[P.qoff + k];
                const float2 q = A.xy[s];
                const BandLine bl = band_line(sm.F, q.x, q.y, d, W, H);
                // whole-image rows accept every valid slot; FP64-only rows send every valid slot to the FP64
                // decision; both use the zero line so that s = 0 for any real keypoint (NaN for empty slots)
                float lo = bl.thr_lo, hi = bl.thr_hi, la0 = bl.a, lb0 = bl.b, lc0 = bl.c;
                if (bl.mode == kBandAll) { lo = INFINITY; hi = INFINITY; la0 = lb0 = lc0 = 0.0f; }
                else if (bl.mode == kBandSlow) { lo = -1.0f; hi = INFINITY; la0 = lb0 = lc0 = 0.0f; }
                L[0] = la0; L[1] = lb0; L[2] = lc0; L[3] = lo; L[4] = hi; L[5] = q.x; L[6] = q.y;
                L[7] = bl.mode == kBandNormal ? bl.t_walk : -1.0f;
                ri[0] = s; ri[1] = A.perm[s]; ri[2] = A.norm[s] * 256; ri[3] = 1;
            } else {
                L[0] = L[1] = L[2] = 0.0f; L[3] = L[4] = -1.0f; L[5] = L[6] = 0.0f; L[7] = -2.0f;
                ri[0] = -1; ri[1] = -1; ri[2] = 0; ri[3] = 0;
            }
        }
        // descriptors of the group: 16*MT rows x 8 chunks of 16 bytes
        for (int e = tid; e < G * 8; e += kThreads) {
            const int r = e >> 3, c = e & 7;
            const int k = q0 + r;
            int4 v = make_int4(0, 0, 0, 0);
            if (k < P.n_a) {
                const int s = qorder[P.qoff + k];
                v = __ldg(reinterpret_cast<const int4 *>(A.desc + (int64_t)s * kDim) + c);
            }
            *reinterpret_cast<int4 *>(&sm.qdesc[r][c * 16]) = v;
        }
        __syncthreads();

        // ---- 2. walk orientation and chord envelope of the group's strips (warp 0)
        if (warp == 0) {
            int votes = 0, nnorm = 0, full = 0;
            for (int r = lane; r < G; r += 32) {
                const float *L = sm.ln[r];
                if (L[7] >= 0.0f) { ++nnorm; votes += fabsf(L[1]) >= fabsf(L[0]); }
                else if (L[7] == -1.0f) full = 1;     // whole-image row (d = inf or FP64-only line)
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                votes += __shfl_xor_sync(0xffffffffu, votes, o);
                nnorm += __shfl_xor_sync(0xffffffffu, nnorm, o);
                full |= __shfl_xor_sync(0xffffffffu, full, o);
            }
            const int colwise = 2 * votes >= nnorm;
            const float ulim = colwise ? W : H;
            float t0 = -INFINITY, t1 = -INFINITY, b0 = INFINITY, b1 = INFINITY, pad = 0.0f;
            for (int r = lane; r < G; r += 32) {
                const float *L = sm.ln[r];
                if (!(L[7] >= 0.0f)) continue;
                float pa = colwise ? L[0] : L[1], pb = colwise ? L[1] : L[0], c = L[2];
                if (pb < 0.0f) { pa = -pa; pb = -pb; c = -c; }
                const float T = L[7];
                if (!(pb > 1e-30f)) { full = 1; continue; }
                const float ib = 1.0f / pb;
                const float e0 = -c * ib, e1 = -fmaf(pa, ulim, c) * ib, h = T * ib;
                t0 = fmaxf(t0, e0 + h); t1 = fmaxf(t1, e1 + h);
                b0 = fminf(b0, e0 - h); b1 = fminf(b1, e1 - h);
                pad = fmaxf(pad, 8.0f * kU * (fabsf(pa) * ulim + fabsf(c) + T) * ib);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                t0 = fmaxf(t0, __shfl_xor_sync(0xffffffffu, t0, o));
                t1 = fmaxf(t1, __shfl_xor_sync(0xffffffffu, t1, o));
                b0 = fminf(b0, __shfl_xor_sync(0xffffffffu, b0, o));
                b1 = fminf(b1, __shfl_xor_sync(0xffffffffu, b1, o));
                pad = fmaxf(pad, __shfl_xor_sync(0xffffffffu, pad, o));
                full |= __shfl_xor_sync(0xffffffffu, full, o);
            }
            if (lane == 0) {
                pad += 1e-3f + 4.0f * kU * (fabsf(t0) + fabsf(t1) + fabsf(b0) + fabsf(b1));
                sm.env[0] = t0 + pad; sm.env[1] = t1 + pad; sm.env[2] = b0 - pad; sm.env[3] = b1 - pad;
                const bool fin = isfinite(sm.env[0]) && isfinite(sm.env[1]) && isfinite(sm.env[2]) &&
                                 isfinite(sm.env[3]);
                sm.walk_full = full || (nnorm > 0 && !fin);
                sm.colwise = colwise;
                if (nnorm == 0 && !full) sm.walk_full = -1;   // nothing to match in this group
            }
        }
        // A fragments of the group (registers for the whole stream)
        int afr[MT][4][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const int8_t *r0 = sm.qdesc[16 * mt + g] + ks * 32 + 4 * t4;
                const int8_t *r1 = sm.qdesc[16 * mt + g + 8] + ks * 32 + 4 * t4;
                afr[mt][ks][0] = *reinterpret_cast<const int *>(r0);
                afr[mt][ks][1] = *reinterpret_cast<const int *>(r1);
                afr[mt][ks][2] = *reinterpret_cast<const int *>(r0 + 16);
                afr[mt][ks][3] = *reinterpret_cast<const int *>(r1 + 16);
            }
        __syncthreads();
        const int walk_full = sm.walk_full;
        const int colwise = walk_full ? 1 : sm.colwise;
        // per-lane row state: rows g and g + 8 of every m-tile
        float la[MT][2], lb[MT][2], lc[MT][2], llo[MT][2], lhi[MT][2];
        int lR[MT][2];
        Top2Key top[MT][2];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = 16 * mt + g + 8 * h;
                la[mt][h] = sm.ln[r][0]; lb[mt][h] = sm.ln[r][1]; lc[mt][h] = sm.ln[r][2];
                llo[mt][h] = sm.ln[r][3]; lhi[mt][h] = sm.ln[r][4];
                lR[mt][h] = sm.rinfo[r][2];
                top[mt][h] = Top2Key{INT_MAX, INT_MAX, 0, 0};
            }

        if (walk_full >= 0) {
            const float cs = (float)(1 << B.cell_shift), inv_cs = 1.0f / cs;
            const int nlines = walk_full ? 1 : (colwise ? B.gx : B.gy);
            const int ng = colwise ? B.gy : B.gx;
            const float ulim = colwise ? W : H, vlim = colwise ? H : W;
            const int32_t *offs = colwise ? B.col_off : B.row_off;
            const float2 *pts = colwise ? B.xy : B.xy_r;
            const float et0 = sm.env[0], et1 = sm.env[1], eb0 = sm.env[2], eb1 = sm.env[3];
            for (int base = 0; base < nlines; base += kMaxRuns) {
                // ---- runs of this pass: one per grid line (or the whole image)
                const int nr = min(kMaxRuns, nlines - base);
                for (int r = tid; r < kMaxRuns; r += kThreads) {
                    int start = 0, len = 0;
                    if (r < nr) {
                        if (walk_full) {
                            start = 0;
                            len = B.n;
                        } else {
                            const int k = base + r;
                            const float u0 = (float)k * cs, u1 = fminf(u0 + cs, ulim);
                            const float f0 = u0 / ulim, f1 = u1 / ulim;
                            const float top0 = fmaf(et1 - et0, f0, et0), top1 = fmaf(et1 - et0, f1, et0);
                            const float bot0 = fmaf(eb1 - eb0, f0, eb0), bot1 = fmaf(eb1 - eb0, f1, eb0);
                            const float lo = fminf(bot0, bot1), hi = fmaxf(top0, top1);
                            if (hi >= 0.0f && lo < vlim) {
                                const int c0 = max(0, (int)floorf(fmaxf(lo, 0.0f) * inv_cs));
                                const int c1 = min(ng - 1, (int)floorf(fminf(hi, vlim) * inv_cs));
                                if (c0 <= c1) {
                                    const int32_t *o = offs + (int64_t)k * ng;
                                    start = o[c0];
                                    len = o[c1 + 1] - start;
                                }
                            }
                        }
                    }
                    sm.run_start[r] = start;
                    sm.run_excl[r] = len;   // lengths for now
                }
                __syncthreads();
                if (warp == 0) {   // exclusive scan of the kMaxRuns lengths
                    int carry = 0;
                    for (int c = 0; c < kMaxRuns; c += 32) {
                        const int v = sm.run_excl[c + lane];
                        int incl = v;
#pragma unroll
                        for (int s = 1; s < 32; s <<= 1) {
                            const int u = __shfl_up_sync(0xffffffffu, incl, s);
                            if (lane >= s) incl += u;
                        }
                        sm.run_excl[c + lane] = carry + incl - v;
                        carry += __shfl_sync(0xffffffffu, incl, 31);
                    }
                    if (lane == 0) sm.run_excl[kMaxRuns] = carry;
                }
                __syncthreads();
                const int total = sm.run_excl[kMaxRuns];
                my_exam += tid == 0 ? (unsigned long long)total * G : 0ull;
                const int nchunks = (total + kN - 1) / kN;

                // loader: 2 threads per slot, each copies 64 bytes of the row
                auto load_chunk = [&](int c, int buf) {
                    const int slot = tid >> 1, half = tid & 1;
                    const int p = c * kN + slot;
                    if (p < total) {
                        int pos = p;                 // whole-image walk: one run starting at 0
                        if (!walk_full) {
                            int lo = 0, hi = kMaxRuns;   // largest r with run_excl[r] <= p
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (sm.run_excl[mid] <= p) lo = mid;
                                else hi = mid;
                            }
                            pos = sm.run_start[lo] + (p - sm.run_excl[lo]);
                        }
                        const int cp = colwise ? pos : B.idx_r[pos];
                        const int4 *src = reinterpret_cast<const int4 *>(B.desc + (int64_t)cp * kDim) + 4 * half;
                        int8_t *dst = sm.bdesc[buf][slot] + 64 * half;
#pragma unroll
                        for (int q = 0; q < 4; ++q) cp_async16(dst + 16 * q, src + q);
                        if (half == 0) {
                            cp_async8(&sm.bxy[buf][slot], pts + pos);
                            cp_async4(&sm.bnb[buf][slot], B.norm + cp);
                            sm.bpos[buf][slot] = cp;
                        }
                    } else if (half == 0) {
                        sm.bxy[buf][slot] = make_float2(__int_as_float(0x7fc00000), 0.0f);   // NaN: never inside
                        sm.bnb[buf][slot] = 0;
                        sm.bpos[buf][slot] = 0;
                    }
                    cp_async_commit();
                };

                // ring of kStages chunks: chunk c lives in stage c % kStages; one group committed per chunk slot
#pragma unroll
                for (int c = 0; c < kStages - 1; ++c) {
                    if (c < nchunks) load_chunk(c, c);
                    else cp_async_commit();
                }
                for (int c = 0; c < nchunks; ++c) {
                    const int buf = c % kStages;
                    cp_async_wait<kStages - 2>();   // chunk c has landed (for this thread's copies)
                    __syncthreads();                // ... for every thread's copies; stage (c-1) is free again
                    if (c + kStages - 1 < nchunks) load_chunk(c + kStages - 1, (c + kStages - 1) % kStages);
                    else cp_async_commit();
                    const int valid_cols = min(kN, total - c * kN);
                    // ---- MMA: this warp's 16 columns = n-tiles 2*warp and 2*warp + 1
                    int acc[MT][2][4];
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int j = 0; j < 2; ++j)
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[mt][j][e] = 0;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const int8_t *br = sm.bdesc[buf][16 * warp + 8 * j + g] + ks * 32 + 4 * t4;
                            const int b0 = *reinterpret_cast<const int *>(br);
                            const int b1 = *reinterpret_cast<const int *>(br + 16);
#pragma unroll
                            for (int mt = 0; mt < MT; ++mt) mma_s8(acc[mt][j], afr[mt][ks], b0, b1);
                        }
                    }
                    // ---- epilogue
                    int k1_before[MT][2];
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int h = 0; h < 2; ++h) k1_before[mt][h] = top[mt][h].k1;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        if (16 * warp + 8 * j >= valid_cols) continue;   // n-tile past the end of the stream
                        const int col = 16 * warp + 8 * j + 2 * t4;
                        const float4 xy2 = *reinterpret_cast<const float4 *>(&sm.bxy[buf][col]);
                        const int2 nb2 = *reinterpret_cast<const int2 *>(&sm.bnb[buf][col]);
                        const int cb0 = nb2.x * 256 + col, cb1 = nb2.y * 256 + col + 1;
#pragma unroll
                        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                            for (int h = 0; h < 2; ++h)
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    const float x = e ? xy2.z : xy2.x, y = e ? xy2.w : xy2.y;
                                    const float s = fmaf(la[mt][h], x, fmaf(lb[mt][h], y, lc[mt][h]));
                                    const float as = fabsf(s);
                                    bool inb = as <= llo[mt][h];
                                    if (!inb && as <= lhi[mt][h]) {
                                        const int r = 16 * mt + g + 8 * h;
                                        inb = band_exact_call(sm.F, sm.ln[r][5], sm.ln[r][6], d, x, y);
                                        ++my_redec;
                                    }
                                    const int key = lR[mt][h] + (e ? cb1 : cb0) - 512 * acc[mt][j][2 * h + e];
                                    const int km = inb ? key : INT_MAX;
                                    Top2Key &T = top[mt][h];
                                    T.k2 = min(T.k2, max(T.k1, km));
                                    T.k1 = min(T.k1, km);
                                    T.cnt += inb;
                                }
                    }
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            if (top[mt][h].k1 < k1_before[mt][h]) top[mt][h].j1 = sm.bpos[buf][top[mt][h].k1 & 255];
                }
                cp_async_wait<0>();
                __syncthreads();
            }
        }

        // ---- 6. merge the top-2 states: quad (4 lanes per row), then the 4 warps
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                Top2Key &T = top[mt][h];
#pragma unroll
                for (int o = 1; o <= 2; o <<= 1) {
                    const int ok1 = __shfl_xor_sync(0xffffffffu, T.k1, o);
                    const int ok2 = __shfl_xor_sync(0xffffffffu, T.k2, o);
                    const int oj1 = __shfl_xor_sync(0xffffffffu, T.j1, o);
                    const int oc = __shfl_xor_sync(0xffffffffu, T.cnt, o);
                    merge_top2(T, ok1, ok2, oj1, oc);
                }
                if (t4 == 0) {
                    int32_t *rd = sm.red[warp][16 * mt + g + 8 * h];
                    rd[0] = T.k1; rd[1] = T.k2; rd[2] = T.j1; rd[3] = T.cnt;
                }
            }
        __syncthreads();
        if (tid < G && sm.rinfo[tid][3]) {
            Top2Key T{INT_MAX, INT_MAX, 0, 0};
#pragma unroll
            for (int w = 0; w < kWarps; ++w) merge_top2(T, sm.red[w][tid][0], sm.red[w][tid][1], sm.red[w][tid][2],
                                                        sm.red[w][tid][3]);
            const int64_t D1 = T.k1 >> 8, D2 = T.k2 >> 8;
            int out = -1;
            if (T.cnt >= 2 && (int64_t)P.q * P.q * D1 < (int64_t)P.p * P.p * D2) out = B.perm[T.j1];
            match_j[P.qoff + sm.rinfo[tid][1]] = out;
            my_cand += (unsigned long long)T.cnt;
        }
    }
    // ---- counters
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_cand += __shfl_xor_sync(0xffffffffu, my_cand, o);
        my_exam += __shfl_xor_sync(0xffffffffu, my_exam, o);
        my_redec += __shfl_xor_sync(0xffffffffu, my_redec, o);
    }
    if (lane == 0) {
        atomicAdd(&sm.stat[0], my_cand);
        atomicAdd(&sm.stat[1], my_exam);
        atomicAdd(&sm.stat[2], my_redec);
    }
    __syncthreads();
    if (tid == 0) {
        BatchCounters *c = ctr + (blockIdx.x % kCounterShards);
        atomicAdd(&c->candidates, sm.stat[0]);
        atomicAdd(&c->examined, sm.stat[1]);
        atomicAdd(&c->redecided, sm.stat[2]);
    }
}

template <int MT>
cudaError_t prepare()
{
    static cudaError_t once = [] {
        cudaError_t e = cudaFuncSetAttribute(match_mma_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(Smem<MT>));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(match_mma_kernel<MT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        return e;
    }();
    return once;
}

template <int MT>
int blocks_per_sm()
{
    int nb = 0;
    if (prepare<MT>() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, match_mma_kernel<MT>, kThreads, sizeof(Smem<MT>)) !=
            cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return std::max(nb, 1);
}

}  // namespace

int match_mma_blocks_per_sm(int mt) { return mt == 2 ? blocks_per_sm<2>() : blocks_per_sm<1>(); }

cudaError_t launch_match_mma(int mt, const ImageDev *imgs, const PairDev *pairs, const int64_t *item_off,
                             int32_t n_pairs, const int32_t *qorder, int64_t item_begin, int64_t item_end,
                             int32_t grid, int32_t *next, int32_t *match_j, BatchCounters *ctr, cudaStream_t st)
{
    const int64_t n = item_end - item_begin;
    if (n <= 0) return cudaSuccess;
    const int persistent = grid > 0;
    const int64_t gsz = persistent ? std::min<int64_t>(grid, n) : n;
    if (mt == 2) {
        cudaError_t e = prepare<2>();
        if (e != cudaSuccess) return e;
        match_mma_kernel<2><<<(unsigned)gsz, kThreads, sizeof(Smem<2>), st>>>(
            imgs, pairs, item_off, n_pairs, qorder, item_begin, item_end, persistent, next, match_j, ctr);
    } else {
        cudaError_t e = prepare<1>();
        if (e != cudaSuccess) return e;
        match_mma_kernel<1><<<(unsigned)gsz, kThreads, sizeof(Smem<1>), st>>>(
            imgs, pairs, item_off, n_pairs, qorder, item_begin, item_end, persistent, next, match_j, ctr);
    }
    return cudaGetLastError();
}

}  // namespace gm
