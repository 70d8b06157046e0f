// gm_approx.cu -- gm_match_pairs_approx: the paper's approximate geometry-aware matching (Sec. 6.2.1 grid-based
// search over four overlapping grids with centre-most cells, Sec. 6.2.2 groups of queries with nearly the same
// epipolar line sharing one candidate set, App. A Steps 1-4), kept next to the exact path for its recall / speed
// trade-off.
//
// The geometry is FP32 with every operation rounded in a fixed order (__fmul_rn, __fadd_rn, __fsub_rn, __fdiv_rn,
// __fsqrt_rn: nothing is contracted), so the integer decisions it takes -- chord ends, sort keys, groups, the cell
// of every sample -- are those of the same FP32 arithmetic anywhere.  For a pair with cell half-size h:
//   Step 1  bin_count / scan / bin_scatter: B's points into the four grids of 2h cells offset by 0 / h (one job per
//           distinct (B, h) of the batch);
//   Step 2  keys: every query's line F (x, y, 1), its chord in B and the chord ends' positions t1 <= t2 along the
//           border; a counting sort on floor(t1) and an in-bin sort by (t1, t2, index); one block per pair walks the
//           sorted keys and marks a group leader wherever t1 or t2 leaves the 2 px window of the current leader;
//   Step 3  one warp per group: the K + 1 equidistant points of the leader's chord (K = ceil(|AB| / h)), for each
//           the cell with the nearest centre among its four cells, every point binned there into a shared-memory
//           bitmap over B's points (C' as a set), each newly set bit also appended to a list of C';
//   Step 4  the same warp: exact squared distances from each query of the group to every point of C' (16 queries x
//           8 candidates per mma.sync.m16n8k32 over the recentred int8 descriptors), top-2, ratio test
//           q^2 D1 < p^2 D2 with |C'| >= 2.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#include "gm_ctx.h"

namespace gm {
namespace {

struct ApproxJob {              // Step 1: grids of one target image for one cell half-size
    const float2 *xy;           // B's points, column-major order
    int32_t n;
    float h, h2, inv_h2;        // cell half-size, cell size 2h, and 1 / 2h when 2h is a power of two
    int32_t pow2;               // 2h is a power of two: dividing by it is the exact scaling by inv_h2
    int32_t nx, ny;             // cells per grid row / column (cell index + 1)
    int64_t cell_base;          // first of this job's 4 * nx * ny cells
};

struct ApproxPair {
    int32_t a, b;               // image slots
    float F[9];
    float h;                    // cell half-size
    float W, H;                 // size of B
    int32_t p, q;
    int32_t n_a, n_b;
    int32_t nbins;              // key bins: floor(t1) in [0, nbins - 2], queries without a chord in nbins - 1
    int32_t job;
    int64_t qoff;               // first query of the pair (global)
    int64_t bin_base;           // first key bin of the pair (global)
};

struct ApproxCounters {
    unsigned long long candidates, cells, bad;
};

// ---------------------------------------------------------------- FP32 geometry (fixed operation order)

__device__ __forceinline__ void line32(const float *F, float x, float y, float &a, float &b, float &c)
{
    a = __fadd_rn(__fadd_rn(__fmul_rn(F[0], x), __fmul_rn(F[1], y)), F[2]);
    b = __fadd_rn(__fadd_rn(__fmul_rn(F[3], x), __fmul_rn(F[4], y)), F[5]);
    c = __fadd_rn(__fadd_rn(__fmul_rn(F[6], x), __fmul_rn(F[7], y)), F[8]);
}

// position along the border, counter-clockwise from the origin
__device__ __forceinline__ float border_t(float x, float y, float W, float H)
{
    if (y == 0.0f) return x;
    if (x == W) return __fadd_rn(W, y);
    if (y == H) return __fadd_rn(__fadd_rn(W, H), __fsub_rn(W, x));
    return __fadd_rn(__fadd_rn(__fadd_rn(W, W), H), __fsub_rn(H, y));
}

struct Chord {
    float xa, ya, ta, xb, yb, tb;
    bool ok;
};

// ends of the line inside [0, W] x [0, H], the lower border position first (candidates in the order left, right,
// bottom, top edge; the first of equal positions wins)
__device__ __forceinline__ void chord_add(Chord &r, float x, float y, float W, float H)
{
    const float t = border_t(x, y, W, H);
    if (!r.ok) {
        r.xa = r.xb = x; r.ya = r.yb = y; r.ta = r.tb = t;
        r.ok = true;
        return;
    }
    if (t < r.ta) { r.xa = x; r.ya = y; r.ta = t; }
    if (t > r.tb) { r.xb = x; r.yb = y; r.tb = t; }
}

__device__ __forceinline__ Chord chord32(float a, float b, float c, float W, float H)
{
    Chord r{};
    r.ok = false;
    if (b != 0.0f) {
        const float y0 = __fdiv_rn(-c, b);
        if (0.0f <= y0 && y0 <= H) chord_add(r, 0.0f, y0, W, H);
        const float yW = __fdiv_rn(-__fadd_rn(__fmul_rn(a, W), c), b);
        if (0.0f <= yW && yW <= H) chord_add(r, W, yW, W, H);
    }
    if (a != 0.0f) {
        const float x0 = __fdiv_rn(-c, a);
        if (0.0f <= x0 && x0 <= W) chord_add(r, x0, 0.0f, W, H);
        const float xH = __fdiv_rn(-__fadd_rn(__fmul_rn(b, H), c), a);
        if (0.0f <= xH && xH <= W) chord_add(r, xH, H, W, H);
    }
    return r;
}

__device__ __forceinline__ int samples_k(const Chord &e, float h)
{
    const float dx = __fsub_rn(e.xb, e.xa), dy = __fsub_rn(e.yb, e.ya);
    const float L = __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
    return (int)ceilf(__fdiv_rn(L, h));
}

__device__ __forceinline__ void sample(const Chord &e, int K, int k, float &x, float &y)
{
    if (K == 0) { x = e.xa; y = e.ya; return; }
    const float kf = (float)k, rk = (float)(K - k), Kf = (float)K;
    x = __fdiv_rn(__fadd_rn(__fmul_rn(kf, e.xa), __fmul_rn(rk, e.xb)), Kf);
    y = __fdiv_rn(__fadd_rn(__fmul_rn(kf, e.ya), __fmul_rn(rk, e.yb)), Kf);
}

// v / 2h, correctly rounded: when 2h is a power of two the product with its exact reciprocal is the same value
__device__ __forceinline__ float div_h2(const ApproxJob &J, float v)
{
    return J.pow2 ? __fmul_rn(v, J.inv_h2) : __fdiv_rn(v, J.h2);
}

__device__ __forceinline__ void cell_of(const ApproxJob &J, int g, float x, float y, int &i, int &j)
{
    const float ox = (g & 1) ? J.h : 0.0f, oy = (g >> 1) ? J.h : 0.0f;
    i = (int)floorf(div_h2(J, __fsub_rn(x, ox)));
    j = (int)floorf(div_h2(J, __fsub_rn(y, oy)));
}

// linear cell index of (g, i, j) in a job, or -1 outside the job's grids
__device__ __forceinline__ int64_t cell_index(const ApproxJob &J, int g, int i, int j)
{
    if (i < -1 || j < -1 || i + 1 >= J.nx || j + 1 >= J.ny) return -1;
    return J.cell_base + ((int64_t)g * J.ny + (j + 1)) * J.nx + (i + 1);
}

// The grids share their x offsets pairwise (grids 0, 2: 0; grids 1, 3: h) and their y offsets likewise, so the two
// cell columns, the two cell rows and their squared centre offsets are computed once each.
__device__ __forceinline__ int64_t chosen_cell(const ApproxJob &J, float px, float py)
{
    const float h = J.h;
    int ci[2], cj[2];
    float ex[2], ey[2];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        const float ox = o ? h : 0.0f;
        ci[o] = (int)floorf(div_h2(J, __fsub_rn(px, ox)));
        cj[o] = (int)floorf(div_h2(J, __fsub_rn(py, ox)));
        const float dx = __fsub_rn(px, __fadd_rn(ox, __fmul_rn((float)(2 * ci[o] + 1), h)));
        const float dy = __fsub_rn(py, __fadd_rn(ox, __fmul_rn((float)(2 * cj[o] + 1), h)));
        ex[o] = __fmul_rn(dx, dx);
        ey[o] = __fmul_rn(dy, dy);
    }
    float best = 0.0f;
    int bg = 0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const float d2 = __fadd_rn(ex[g & 1], ey[g >> 1]);
        if (g == 0 || d2 < best) { best = d2; bg = g; }
    }
    return cell_index(J, bg, ci[bg & 1], cj[bg >> 1]);
}

template <typename T>
__device__ __forceinline__ int upper_index(const T *prefix, int n, T v)   // largest k < n with prefix[k] <= v
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- Step 1: grids

__global__ void bin_count_kernel(const ApproxJob *__restrict__ jobs, const int64_t *__restrict__ job_pt, int n_jobs,
                                 int32_t *__restrict__ cnt, ApproxCounters *ctr)
{
    const int64_t total = job_pt[n_jobs];
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total; u += (int64_t)gridDim.x * blockDim.x) {
        const int jb = upper_index(job_pt, n_jobs, u);
        const ApproxJob &J = jobs[jb];
        const float2 p = J.xy[u - job_pt[jb]];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            int i, j;
            cell_of(J, g, p.x, p.y, i, j);
            const int64_t c = cell_index(J, g, i, j);
            if (c < 0) atomicAdd(&ctr->bad, 1ull);
            else atomicAdd(&cnt[c], 1);
        }
    }
}

__global__ void bin_scatter_kernel(const ApproxJob *__restrict__ jobs, const int64_t *__restrict__ job_pt, int n_jobs,
                                   const int32_t *__restrict__ off, int32_t *__restrict__ cursor,
                                   int32_t *__restrict__ members)
{
    const int64_t total = job_pt[n_jobs];
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total; u += (int64_t)gridDim.x * blockDim.x) {
        const int jb = upper_index(job_pt, n_jobs, u);
        const ApproxJob &J = jobs[jb];
        const int32_t pos = (int32_t)(u - job_pt[jb]);
        const float2 p = J.xy[pos];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            int i, j;
            cell_of(J, g, p.x, p.y, i, j);
            const int64_t c = cell_index(J, g, i, j);
            if (c >= 0) members[off[c] + atomicAdd(&cursor[c], 1)] = pos;
        }
    }
}

// ---------------------------------------------------------------- Step 2: keys, order, groups

__global__ void keys_kernel(const ApproxPair *__restrict__ P, const int64_t *__restrict__ qoff, int n_pairs,
                            const ImageDev *__restrict__ imgs, float *__restrict__ T1, float *__restrict__ T2,
                            uint8_t *__restrict__ has, int32_t *__restrict__ bcnt)
{
    const int64_t Q = qoff[n_pairs];
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < Q; u += (int64_t)gridDim.x * blockDim.x) {
        const int k = upper_index(qoff, n_pairs, u);
        const ApproxPair &pr = P[k];
        const ImageDev &A = imgs[pr.a];
        const int32_t i = (int32_t)(u - qoff[k]);
        const float2 pt = A.xy[A.inv_perm[i]];
        float a, b, c;
        line32(pr.F, pt.x, pt.y, a, b, c);
        const Chord e = chord32(a, b, c, pr.W, pr.H);
        T1[u] = e.ok ? e.ta : 0.0f;
        T2[u] = e.ok ? e.tb : 0.0f;
        has[u] = e.ok ? 1 : 0;
        const int bin = e.ok ? min((int)floorf(e.ta), pr.nbins - 2) : pr.nbins - 1;
        atomicAdd(&bcnt[pr.bin_base + bin], 1);
    }
}

__global__ void key_scatter_kernel(const ApproxPair *__restrict__ P, const int64_t *__restrict__ qoff, int n_pairs,
                                   const float *__restrict__ T1, const uint8_t *__restrict__ has,
                                   const int32_t *__restrict__ boff, int32_t *__restrict__ bcur,
                                   int32_t *__restrict__ order)
{
    const int64_t Q = qoff[n_pairs];
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < Q; u += (int64_t)gridDim.x * blockDim.x) {
        const int k = upper_index(qoff, n_pairs, u);
        const ApproxPair &pr = P[k];
        const int bin = has[u] ? min((int)floorf(T1[u]), pr.nbins - 2) : pr.nbins - 1;
        const int64_t gb = pr.bin_base + bin;
        order[boff[gb] + atomicAdd(&bcur[gb], 1)] = (int32_t)(u - qoff[k]);
    }
}

// (t1, t2, index) order inside every key bin (insertion sort: bins hold a few queries); the bin of queries without
// a chord keeps any order, since each of them is a group of its own
__global__ void bin_sort_kernel(const ApproxPair *__restrict__ P, const int64_t *__restrict__ bin_pre, int n_pairs,
                                const int32_t *__restrict__ boff, const float *__restrict__ T1,
                                const float *__restrict__ T2, int32_t *__restrict__ order)
{
    const int64_t NB = bin_pre[n_pairs];
    for (int64_t gb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gb < NB; gb += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s0 = boff[gb], s1 = boff[gb + 1];
        if (s1 - s0 < 2) continue;
        const int k = upper_index(bin_pre, n_pairs, gb);
        const ApproxPair &pr = P[k];
        if (gb - pr.bin_base == pr.nbins - 1) continue;
        const float *t1 = T1 + pr.qoff, *t2 = T2 + pr.qoff;
        for (int32_t s = s0 + 1; s < s1; ++s) {
            const int32_t v = order[s];
            const float a1 = t1[v], a2 = t2[v];
            int32_t r = s - 1;
            while (r >= s0) {
                const int32_t w = order[r];
                const bool after = t1[w] > a1 || (t1[w] == a1 && (t2[w] > a2 || (t2[w] == a2 && w > v)));
                if (!after) break;
                order[r + 1] = w;
                --r;
            }
            order[r + 1] = v;
        }
    }
}

constexpr int kWalkWin = 4096;      // sorted keys per shared-memory window of the group walk

// One block per pair: warp 0 walks the sorted keys and flags every group leader (flag[s] = 1 at sorted position s).
__global__ void group_walk_kernel(const ApproxPair *__restrict__ P, const int32_t *__restrict__ order,
                                  const float *__restrict__ T1, const float *__restrict__ T2,
                                  const uint8_t *__restrict__ has, int32_t *__restrict__ flag)
{
    __shared__ float w1[kWalkWin], w2[kWalkWin];
    __shared__ uint8_t wh[kWalkWin];
    const ApproxPair &pr = P[blockIdx.x];
    const int64_t q0 = pr.qoff;
    const int32_t n = pr.n_a;
    float l1 = 0.0f, l2 = 0.0f;
    bool lh = false;
    for (int32_t base = 0; base < n; base += kWalkWin) {
        const int32_t cnt = min(kWalkWin, n - base);
        __syncthreads();
        for (int32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int64_t u = q0 + order[q0 + base + t];
            w1[t] = T1[u];
            w2[t] = T2[u];
            wh[t] = has[u];
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int32_t s = 0;
            if (base == 0) {   // the pair's first query leads the first group
                if (lane == 0) flag[q0] = 1;
                l1 = w1[0]; l2 = w2[0]; lh = wh[0] != 0;
                s = 1;
            }
            while (s < cnt) {
                const int32_t pos = s + lane;
                bool viol = false;
                if (pos < cnt)
                    viol = !wh[pos] || !lh || fabsf(__fsub_rn(w1[pos], l1)) > 2.0f || fabsf(__fsub_rn(w2[pos], l2)) > 2.0f;
                const unsigned bal = __ballot_sync(0xffffffffu, viol);
                if (!bal) { s += 32; continue; }
                const int32_t first = s + __ffs(bal) - 1;
                if (lane == 0) flag[q0 + base + first] = 1;
                l1 = w1[first]; l2 = w2[first]; lh = wh[first] != 0;
                s = first + 1;
            }
        }
    }
}

__global__ void group_start_kernel(const int32_t *__restrict__ flag, const int32_t *__restrict__ gid, int64_t Q,
                                   int32_t *__restrict__ gstart)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < Q; s += (int64_t)gridDim.x * blockDim.x)
        if (flag[s]) gstart[gid[s]] = (int32_t)s;
    if (blockIdx.x == 0 && threadIdx.x == 0) gstart[gid[Q]] = (int32_t)Q;
}

// ---------------------------------------------------------------- Steps 3-4: one warp per group

constexpr int kQTile = 16;           // queries of a group scored together (the mma m dimension)
constexpr int kSampleBatch = 8;      // chord samples a lane looks up at a time
constexpr int kListCap = 512;        // candidate positions in the list: the sampled C', or one round of compaction
constexpr int kRoundWords = kListCap / 32;   // bitmap words per compaction round: they hold at most kListCap bits
static_assert(kListCap % 32 == 0 && kRoundWords >= 1 && kRoundWords <= 32, "a round must fit an empty list");
constexpr size_t kWarpExtra = kQTile * kDim + 4 * kListCap + 4 * kQTile + 16;   // query rows, list, query norms, count

__device__ __forceinline__ void mma_s8(int (&d)[4], const int (&a)[4], int b0, int b1)
{
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
constexpr int kMatchThreads = 128;
constexpr int kMatchMinBlocks = 8;   // resident blocks per SM that __launch_bounds__ asks the register allocation for
constexpr int kWarpsPerBlock = 4;    // groups (one warp each) per block of the match kernel, at most kMatchThreads / 32

__global__ void __launch_bounds__(kMatchThreads, kMatchMinBlocks) approx_match_kernel(const ApproxPair *__restrict__ P, const int64_t *__restrict__ qoff, int n_pairs,
                                    const ApproxJob *__restrict__ jobs, const ImageDev *__restrict__ imgs,
                                    const int32_t *__restrict__ cell_off, const int32_t *__restrict__ members,
                                    const int32_t *__restrict__ order, const uint8_t *__restrict__ has,
                                    const int32_t *__restrict__ gstart, int64_t G, int32_t words,
                                    int32_t *__restrict__ match_j, ApproxCounters *ctr)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * wpb + wib;
    if (g >= G) return;
    uint32_t *bm = reinterpret_cast<uint32_t *>(sm + (size_t)wib * ((size_t)words * 4 + kWarpExtra));
    int8_t *qd = reinterpret_cast<int8_t *>(bm + words);
    const int32_t s0 = gstart[g], s1 = gstart[g + 1];
    const int k = upper_index(qoff, n_pairs, (int64_t)s0);
    const ApproxPair &pr = P[k];
    const ImageDev &A = imgs[pr.a], &B = imgs[pr.b];
    const ApproxJob &J = jobs[pr.job];
    const int64_t q0 = pr.qoff;
    const int32_t lead = order[s0];
    // Step 3: C' of the leader's chord as a bitmap over B's column-major positions
    // every newly set bit also appends its position to the candidate list (up to kListCap entries; the count goes
    // on, and a longer C' is compacted from the bitmap round by round below)
    const int32_t nw = (pr.n_b + 31) >> 5;
    int32_t *list = reinterpret_cast<int32_t *>(qd + kQTile * kDim);
    int32_t *qn_s = list + kListCap;
    int32_t *nl_s = qn_s + kQTile;
    for (int32_t w = lane; w < nw; w += 32) bm[w] = 0u;
    if (lane == 0) *nl_s = 0;
    __syncwarp();
    if (has[q0 + lead]) {
        const float2 pt = A.xy[A.inv_perm[lead]];
        float a, b, c;
        line32(pr.F, pt.x, pt.y, a, b, c);
        const Chord e = chord32(a, b, c, pr.W, pr.H);
        const int K = samples_k(e, pr.h);
        for (int base = 0; base <= K; base += 32 * kSampleBatch) {
            // kSampleBatch samples per lane at a time: their cell lookups are independent loads in flight together
            int lo[kSampleBatch], hi[kSampleBatch];
#pragma unroll
            for (int t = 0; t < kSampleBatch; ++t) {
                const int kk = base + lane + 32 * t;
                int64_t cidx = -1;
                if (kk <= K) {
                    float x, y;
                    sample(e, K, kk, x, y);
                    cidx = chosen_cell(J, x, y);
                }
                lo[t] = cidx >= 0 ? __ldg(cell_off + cidx) : 0;
                hi[t] = cidx >= 0 ? __ldg(cell_off + cidx + 1) : 0;
            }
            // the cells' members, one from each of the lane's samples at a time (independent loads in flight
            // together; the bitmap OR does not depend on the order)
            int span = 0;
#pragma unroll
            for (int t = 0; t < kSampleBatch; ++t) span = max(span, hi[t] - lo[t]);
            for (int i = 0; i < span; ++i) {
                int32_t pos[kSampleBatch];
#pragma unroll
                for (int t = 0; t < kSampleBatch; ++t) pos[t] = lo[t] + i < hi[t] ? __ldg(members + lo[t] + i) : -1;
#pragma unroll
                for (int t = 0; t < kSampleBatch; ++t)
                    if (pos[t] >= 0) {
                        const uint32_t bit = 1u << (pos[t] & 31);
                        if (!(atomicOr(&bm[pos[t] >> 5], bit) & bit)) {
                            const int32_t slot = atomicAdd(nl_s, 1);
                            if (slot < kListCap) list[slot] = pos[t];
                        }
                    }
            }
        }
        if (lane == 0) atomicAdd(&ctr->cells, (unsigned long long)(K + 1));
    }
    __syncwarp();
    const int32_t cnt = *reinterpret_cast<volatile int32_t *>(nl_s);   // |C'|
    const bool direct = cnt <= kListCap;                                // the list already holds all of C'
    if (lane == 0) atomicAdd(&ctr->candidates, (unsigned long long)cnt * (unsigned long long)(s1 - s0));
    // Step 4: exact distances from each query of the group to C', top-2, ratio test.  The group's queries are
    // scored 16 at a time against 8 candidates at a time by mma.sync.m16n8k32.s8 (the int32 accumulator holds the
    // exact dot product a'.b') over the list built while sampling; a C' longer than kListCap is compacted from the
    // bitmap instead, kListCap positions per round.
    // Fragments (lane = 4 g + t): A rows g and g + 8, bytes 4t .. 4t + 3 and 16 + 4t .. of each 32-byte K step;
    // B column g (a candidate), the same bytes; accumulator element 2 h + e = (row g + 8 h, column 2 t + e).
    const int gq = lane >> 2, t4 = lane & 3;
    for (int32_t c0 = s0; c0 < s1; c0 += kQTile) {
        const int nq = min(kQTile, s1 - c0);
        __syncwarp();
        for (int t = 0; t < kQTile; ++t) {   // 128 bytes per query row (zeros past the group), one word per lane
            int32_t w = 0;
            if (t < nq) w = reinterpret_cast<const int32_t *>(A.desc + (size_t)A.inv_perm[order[c0 + t]] * kDim)[lane];
            reinterpret_cast<int32_t *>(qd + t * kDim)[lane] = w;
        }
        if (lane < kQTile) qn_s[lane] = lane < nq ? A.norm[A.inv_perm[order[c0 + lane]]] : 0;
        __syncwarp();
        int afr[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const int8_t *r0 = qd + gq * kDim + ks * 32 + 4 * t4;
            const int8_t *r1 = qd + (gq + 8) * kDim + ks * 32 + 4 * t4;
            afr[ks][0] = *reinterpret_cast<const int *>(r0);
            afr[ks][1] = *reinterpret_cast<const int *>(r1);
            afr[ks][2] = *reinterpret_cast<const int *>(r0 + 16);
            afr[ks][3] = *reinterpret_cast<const int *>(r1 + 16);
        }
        const int qn0 = qn_s[gq], qn1 = qn_s[gq + 8];
        int D1[2] = {INT_MAX, INT_MAX}, D2[2] = {INT_MAX, INT_MAX}, J1[2] = {INT_MAX, INT_MAX};
        for (int32_t w0 = 0; w0 < nw;) {
            int32_t nl = 0;
            if (direct) {
                nl = cnt;
                w0 = nw;
            }
            while (w0 < nw) {   // kRoundWords words per round hold at most kListCap bits: every round fits an empty list
                const int32_t w = w0 + lane;
                uint32_t bits = lane < kRoundWords && w < nw ? bm[w] : 0u;
                const int c = __popc(bits);
                int inc = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                const int tot = __shfl_sync(0xffffffffu, inc, 31);
                if (nl + tot > kListCap) break;
                int at = nl + inc - c;
                while (bits) {
                    list[at++] = (w << 5) + __ffs(bits) - 1;
                    bits &= bits - 1u;
                }
                nl += tot;
                w0 += kRoundWords;
            }
            __syncwarp();
            // B fragments of n-tile n0 (8 candidates; padding columns repeat a real one), loaded one tile ahead
            auto load_b = [&](int32_t n0, int (&bf)[8]) {
                const int cj = n0 + gq < nl ? list[n0 + gq] : list[n0];
                const int8_t *brow = B.desc + (size_t)cj * kDim + 4 * t4;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    bf[2 * ks] = __ldg(reinterpret_cast<const int *>(brow + ks * 32));
                    bf[2 * ks + 1] = __ldg(reinterpret_cast<const int *>(brow + ks * 32 + 16));
                }
            };
            int bcur[8];
            if (nl > 0) load_b(0, bcur);
            for (int32_t n0 = 0; n0 < nl; n0 += 8) {   // one n-tile of 8 candidates
                int bnext[8];
                if (n0 + 8 < nl) load_b(n0 + 8, bnext);
                int acc[4] = {0, 0, 0, 0};
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) mma_s8(acc, afr[ks], bcur[2 * ks], bcur[2 * ks + 1]);
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int col = n0 + 2 * t4 + e;
                    if (col >= nl) continue;
                    const int j = list[col];
                    const int nb = __ldg(B.norm + j);
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int D = (hh ? qn1 : qn0) + nb - 2 * acc[2 * hh + e];
                        if (D < D1[hh] || (D == D1[hh] && j < J1[hh])) { D2[hh] = D1[hh]; D1[hh] = D; J1[hh] = j; }
                        else if (D < D2[hh]) D2[hh] = D;
                    }
                }
                if (n0 + 8 < nl) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) bcur[u] = bnext[u];
                }
            }
            __syncwarp();
        }
        // merge the top-2 lists of the four lanes of each row pair (t = 0 .. 3)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
            for (int o = 1; o < 4; o <<= 1) {
                const int od1 = __shfl_xor_sync(0xffffffffu, D1[hh], o);
                const int od2 = __shfl_xor_sync(0xffffffffu, D2[hh], o);
                const int oj1 = __shfl_xor_sync(0xffffffffu, J1[hh], o);
                if (od1 < D1[hh] || (od1 == D1[hh] && oj1 < J1[hh])) {
                    D2[hh] = min(D1[hh], od2);
                    D1[hh] = od1;
                    J1[hh] = oj1;
                } else {
                    D2[hh] = min(D2[hh], od1);
                }
            }
        }
        if (t4 == 0) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int t = gq + 8 * hh;
                if (t >= nq) continue;
                const int64_t pp = pr.p, qq = pr.q;
                int out = -1;
                if (cnt >= 2 && qq * qq * (int64_t)D1[hh] < pp * pp * (int64_t)D2[hh]) out = B.perm[J1[hh]];
                match_j[q0 + order[c0 + t]] = out;
            }
        }
    }
}

#define GM_CUDA_A(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return gm::fail(GM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace
}  // namespace gm

extern "C" {

gm_status gm_match_pairs_approx(gm_ctx *ctx, int32_t n_pairs, const gm_pair *pairs, float cell_scale,
                                int64_t *pair_off, int32_t *matches, int64_t cap, int64_t *n_written,
                                gm_approx_stats *stats)
{
    gm::NvtxRange nvtx_("gm_match_pairs_approx");
    using namespace gm;
    const char *fn = "gm_match_pairs_approx";
    if (!ctx || n_pairs < 0 || (n_pairs > 0 && !pairs) || !pair_off || !n_written || cap < 0 || (cap > 0 && !matches) ||
        !(cell_scale > 0.0f) || !std::isfinite(cell_scale))
        return fail(GM_ERR_INVALID, "%s: bad arguments", fn);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA_A(cudaSetDevice(ctx->device));
    *n_written = 0;
    if (stats) *stats = gm_approx_stats{};
    cudaStream_t s = ctx->ws.stream;
    const bool dev_off = is_device_ptr(pair_off);
    if (n_pairs == 0) {
        if (dev_off) GM_CUDA_A(cudaMemset(pair_off, 0, sizeof(int64_t)));
        else pair_off[0] = 0;
        return GM_OK;
    }
    // pairs, jobs (one per distinct (B, h)), key bins
    std::vector<PairDev> pd(n_pairs);
    std::vector<ApproxPair> ap(n_pairs);
    std::vector<int64_t> qoff(n_pairs + 1, 0), bin_pre(n_pairs + 1, 0);
    std::vector<ApproxJob> jobs;
    std::vector<int64_t> job_pt(1, 0);
    std::map<std::pair<int32_t, uint32_t>, int32_t> job_of;
    int64_t cells = 0;
    int32_t max_nb = 0;
    gm_status st;
    for (int32_t k = 0; k < n_pairs; ++k) {
        if ((st = prepare_pair(ctx, pairs[k], k, pd[k])) != GM_OK) return st;
        const float d = pairs[k].band_px;
        volatile float hv = d * cell_scale;   // one IEEE single multiplication
        const float h = hv;
        if (!std::isfinite(d) || !(h >= 0.5f) || !std::isfinite(h))
            return fail(GM_ERR_INVALID, "%s: pair %d: band_px * cell_scale must be finite and >= 0.5 px", fn, k);
        const ImageDev &B = ctx->slots[pd[k].b]->dev;
        if (B.n > (1 << 22)) return fail(GM_ERR_INVALID, "%s: pair %d: more than 2^22 target keypoints", fn, k);
        ApproxPair &a = ap[k];
        a.a = pd[k].a;
        a.b = pd[k].b;
        std::memcpy(a.F, pairs[k].F, sizeof(a.F));
        a.h = h;
        a.W = (float)B.width;
        a.H = (float)B.height;
        a.p = pairs[k].ratio_num;
        a.q = pairs[k].ratio_den;
        a.n_a = pd[k].n_a;
        a.n_b = B.n;
        a.nbins = 2 * (B.width + B.height) + 2;
        uint32_t hb;
        std::memcpy(&hb, &h, 4);
        auto key = std::make_pair(pd[k].b, hb);
        auto it = job_of.find(key);
        if (it == job_of.end()) {
            ApproxJob J{};
            J.xy = B.xy;
            J.n = B.n;
            J.h = h;
            J.h2 = h + h;   // exact: a doubling
            int ex2 = 0;
            J.pow2 = std::frexp(J.h2, &ex2) == 0.5f;
            J.inv_h2 = J.pow2 ? std::ldexp(1.0f, 1 - ex2) : 0.0f;
            J.nx = (int32_t)std::floor((double)B.width / (2.0 * h)) + 3;   // cell index -1 .. floor(W / 2h) + 1
            J.ny = (int32_t)std::floor((double)B.height / (2.0 * h)) + 3;
            J.cell_base = cells;
            cells += 4 * (int64_t)J.nx * J.ny;
            it = job_of.emplace(key, (int32_t)jobs.size()).first;
            jobs.push_back(J);
            job_pt.push_back(job_pt.back() + B.n);
        }
        a.job = it->second;
        a.qoff = qoff[k];
        a.bin_base = bin_pre[k];
        pd[k].qoff = qoff[k];
        qoff[k + 1] = qoff[k] + pd[k].n_a;
        bin_pre[k + 1] = bin_pre[k] + a.nbins;
        max_nb = std::max(max_nb, B.n);
    }
    const int64_t Q = qoff[n_pairs], NB = bin_pre[n_pairs], NJ = (int64_t)jobs.size(), NPT = job_pt.back();
    if (Q == 0) {   // no queries: every pair has an empty match list
        std::vector<int64_t> z(n_pairs + 1, 0);
        if (dev_off) GM_CUDA_A(cudaMemcpy(pair_off, z.data(), 8 * (n_pairs + 1), cudaMemcpyHostToDevice));
        else std::memcpy(pair_off, z.data(), 8 * (n_pairs + 1));
        return GM_OK;
    }
    if (Q > INT32_MAX / 2 || NB > INT32_MAX / 2 || cells > INT32_MAX / 2 || 4 * NPT > INT32_MAX / 2)
        return fail(GM_ERR_INVALID, "%s: batch too large for one call", fn);
    // one device allocation for everything
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += align_up(std::max<size_t>(bytes, 1), 256); return o; };
    const size_t o_pd = take(sizeof(PairDev) * n_pairs), o_ap = take(sizeof(ApproxPair) * n_pairs);
    const size_t o_qoff = take(8 * (n_pairs + 1)), o_bpre = take(8 * (n_pairs + 1));
    const size_t o_jobs = take(sizeof(ApproxJob) * NJ), o_jpt = take(8 * (NJ + 1));
    const size_t o_ccnt = take(4 * (cells + 1)), o_coff = take(4 * (cells + 1)), o_ccur = take(4 * cells);
    const size_t o_mem = take(4 * 4 * NPT), o_bsum = take(4 * ((std::max({cells, NB, Q}) + 1) / 1024 + 2));
    const size_t o_t1 = take(4 * Q), o_t2 = take(4 * Q), o_has = take(Q), o_ord = take(4 * Q);
    const size_t o_bcnt = take(4 * (NB + 1)), o_boff = take(4 * (NB + 1)), o_bcur = take(4 * NB);
    const size_t o_flag = take(4 * (Q + 1)), o_gid = take(4 * (Q + 1)), o_gst = take(4 * (Q + 1));
    const size_t o_mj = take(4 * Q), o_cnt = take(4 * n_pairs), o_off = take(8 * (n_pairs + 1));
    const size_t o_rows = take(8 * Q), o_ctr = take(sizeof(ApproxCounters));
    if ((st = ensure_dev(ctx, ctx->d_approx, off)) != GM_OK) return st;
    char *base = static_cast<char *>(ctx->d_approx.p);
    auto at = [&](size_t o) { return base + o; };
    PairDev *d_pd = reinterpret_cast<PairDev *>(at(o_pd));
    ApproxPair *d_ap = reinterpret_cast<ApproxPair *>(at(o_ap));
    int64_t *d_qoff = reinterpret_cast<int64_t *>(at(o_qoff)), *d_bpre = reinterpret_cast<int64_t *>(at(o_bpre));
    ApproxJob *d_jobs = reinterpret_cast<ApproxJob *>(at(o_jobs));
    int64_t *d_jpt = reinterpret_cast<int64_t *>(at(o_jpt));
    int32_t *ccnt = reinterpret_cast<int32_t *>(at(o_ccnt)), *coff = reinterpret_cast<int32_t *>(at(o_coff));
    int32_t *ccur = reinterpret_cast<int32_t *>(at(o_ccur)), *mem = reinterpret_cast<int32_t *>(at(o_mem));
    int32_t *bsum = reinterpret_cast<int32_t *>(at(o_bsum));
    float *T1 = reinterpret_cast<float *>(at(o_t1)), *T2 = reinterpret_cast<float *>(at(o_t2));
    uint8_t *has = reinterpret_cast<uint8_t *>(at(o_has));
    int32_t *ord = reinterpret_cast<int32_t *>(at(o_ord));
    int32_t *bcnt = reinterpret_cast<int32_t *>(at(o_bcnt)), *boff = reinterpret_cast<int32_t *>(at(o_boff));
    int32_t *bcur = reinterpret_cast<int32_t *>(at(o_bcur));
    int32_t *flag = reinterpret_cast<int32_t *>(at(o_flag)), *gid = reinterpret_cast<int32_t *>(at(o_gid));
    int32_t *gst = reinterpret_cast<int32_t *>(at(o_gst));
    int32_t *mj = reinterpret_cast<int32_t *>(at(o_mj)), *counts = reinterpret_cast<int32_t *>(at(o_cnt));
    int64_t *d_off = reinterpret_cast<int64_t *>(at(o_off));
    int32_t *rows = reinterpret_cast<int32_t *>(at(o_rows));
    ApproxCounters *ctr = reinterpret_cast<ApproxCounters *>(at(o_ctr));
    GM_CUDA_A(cudaMemcpyAsync(d_pd, pd.data(), sizeof(PairDev) * n_pairs, cudaMemcpyHostToDevice, s));
    GM_CUDA_A(cudaMemcpyAsync(d_ap, ap.data(), sizeof(ApproxPair) * n_pairs, cudaMemcpyHostToDevice, s));
    GM_CUDA_A(cudaMemcpyAsync(d_qoff, qoff.data(), 8 * (n_pairs + 1), cudaMemcpyHostToDevice, s));
    GM_CUDA_A(cudaMemcpyAsync(d_bpre, bin_pre.data(), 8 * (n_pairs + 1), cudaMemcpyHostToDevice, s));
    GM_CUDA_A(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(ApproxJob) * NJ, cudaMemcpyHostToDevice, s));
    GM_CUDA_A(cudaMemcpyAsync(d_jpt, job_pt.data(), 8 * (NJ + 1), cudaMemcpyHostToDevice, s));
    GM_CUDA_A(cudaMemsetAsync(ccnt, 0, 4 * (cells + 1), s));
    GM_CUDA_A(cudaMemsetAsync(ccur, 0, 4 * std::max<int64_t>(cells, 1), s));
    GM_CUDA_A(cudaMemsetAsync(bcnt, 0, 4 * (NB + 1), s));
    GM_CUDA_A(cudaMemsetAsync(bcur, 0, 4 * NB, s));
    GM_CUDA_A(cudaMemsetAsync(flag, 0, 4 * (Q + 1), s));
    GM_CUDA_A(cudaMemsetAsync(ctr, 0, sizeof(ApproxCounters), s));
    const int grid = std::max(1, ctx->num_sms * 8);
    // Step 1
    bin_count_kernel<<<grid, 256, 0, s>>>(d_jobs, d_jpt, (int)NJ, ccnt, ctr);
    GM_CUDA_A(launch_exclusive_scan(ccnt, (int32_t)cells, coff, bsum, s));
    bin_scatter_kernel<<<grid, 256, 0, s>>>(d_jobs, d_jpt, (int)NJ, coff, ccur, mem);
    // Step 2
    keys_kernel<<<grid, 256, 0, s>>>(d_ap, d_qoff, n_pairs, static_cast<const ImageDev *>(ctx->d_imgs.p), T1, T2, has,
                                     bcnt);
    GM_CUDA_A(launch_exclusive_scan(bcnt, (int32_t)NB, boff, bsum, s));
    key_scatter_kernel<<<grid, 256, 0, s>>>(d_ap, d_qoff, n_pairs, T1, has, boff, bcur, ord);
    bin_sort_kernel<<<grid, 256, 0, s>>>(d_ap, d_bpre, n_pairs, boff, T1, T2, ord);
    group_walk_kernel<<<n_pairs, 128, 0, s>>>(d_ap, ord, T1, T2, has, flag);
    GM_CUDA_A(launch_exclusive_scan(flag, (int32_t)Q, gid, bsum, s));
    group_start_kernel<<<grid, 256, 0, s>>>(flag, gid, Q, gst);
    GM_CUDA_A(cudaGetLastError());
    int32_t G = 0;
    GM_CUDA_A(cudaMemcpyAsync(&G, gid + Q, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GM_CUDA_A(cudaStreamSynchronize(s));
    // Steps 3-4
    const int32_t words = ((max_nb + 31) / 32 + 3) & ~3;   // a multiple of 4 words keeps the query rows 16-byte aligned
    const size_t per_warp = (size_t)words * 4 + kWarpExtra;
    int wpb = kWarpsPerBlock;
    while (wpb > 1 && per_warp * wpb > 200 * 1024) --wpb;
    if (per_warp * wpb > 200 * 1024) return fail(GM_ERR_INVALID, "%s: target image too large for the bitmap", fn);
    const size_t smem = per_warp * wpb;
    if (smem > 48 * 1024)
        GM_CUDA_A(cudaFuncSetAttribute(approx_match_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (G > 0)
        approx_match_kernel<<<(unsigned)((G + wpb - 1) / wpb), 32 * wpb, smem, s>>>(
            d_ap, d_qoff, n_pairs, d_jobs, static_cast<const ImageDev *>(ctx->d_imgs.p), coff, mem, ord, has, gst, G,
            words, mj, ctr);
    GM_CUDA_A(cudaGetLastError());
    GM_CUDA_A(launch_count_matches(d_pd, n_pairs, mj, counts, d_off, s));
    GM_CUDA_A(launch_write_matches(d_pd, n_pairs, mj, d_off, rows, s));
    std::vector<int64_t> h_off(n_pairs + 1);
    ApproxCounters hc{};
    GM_CUDA_A(cudaMemcpyAsync(h_off.data(), d_off, 8 * (n_pairs + 1), cudaMemcpyDeviceToHost, s));
    GM_CUDA_A(cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
    GM_CUDA_A(cudaStreamSynchronize(s));
    if (hc.bad) return fail(GM_ERR_INVALID, "%s: %llu keypoints outside their grids", fn, hc.bad);
    if (stats) {
        stats->n_groups = G;
        stats->n_candidates = (int64_t)hc.candidates;
        stats->n_cells = (int64_t)hc.cells;
    }
    const int64_t total = h_off[n_pairs];
    *n_written = total;
    if (dev_off) GM_CUDA_A(cudaMemcpyAsync(pair_off, d_off, 8 * (n_pairs + 1), cudaMemcpyDeviceToDevice, s));
    else std::memcpy(pair_off, h_off.data(), 8 * (n_pairs + 1));
    if (total > cap) {
        GM_CUDA_A(cudaStreamSynchronize(s));
        return fail(GM_ERR_NOMEM, "%s: %lld matches exceed cap %lld", fn, (long long)total, (long long)cap);
    }
    if (total > 0) GM_CUDA_A(cudaMemcpyAsync(matches, rows, 8 * total, cudaMemcpyDefault, s));
    GM_CUDA_A(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // extern "C"
