// gm_match_simt.cu -- SIMT matching path: one warp per query (App. A Steps 3-4 fused into one kernel).
//
// The warp walks the query's band over B's grid (gm_band.cuh); lanes test visited points 32 at a time, the
// inside points are compacted into a per-warp queue in shared memory, and every 32 queued candidates each lane
// computes one exact squared distance D = |a|^2 + |b|^2 - 2 a.b with 32 dp4a over the recentred int8
// descriptors (a - 128, b - 128 give the same differences as a, b).  Each lane keeps a running top-2; a warp
// shuffle merges them and lane 0 applies the integer ratio test q^2 D1 < p^2 D2 (Sec. 2.3, App. A Step 4).
//
// Ties: with p < q, equal nearest distances make D1 == D2 and the strict test rejects, so which of the tied
// candidates is called "nearest" never reaches the output; only the strict minimum's index is kept.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "gm_band.cuh"
#include "gm_internal.h"

namespace gm {
namespace {

constexpr int kWarpsPerBlock = kQueriesPerItem;
constexpr int kCounterShards = 64;

struct Top2 {
    int d1, d2, j1;
};

__device__ __forceinline__ void top2_push(Top2 &t, int D, int j)
{
    if (D < t.d1) { t.d2 = t.d1; t.d1 = D; t.j1 = j; }
    else if (D < t.d2) { t.d2 = D; }
}

__device__ __forceinline__ Top2 top2_warp_merge(Top2 t)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int od1 = __shfl_xor_sync(0xffffffffu, t.d1, o);
        const int od2 = __shfl_xor_sync(0xffffffffu, t.d2, o);
        const int oj1 = __shfl_xor_sync(0xffffffffu, t.j1, o);
        const int nd2 = min(max(t.d1, od1), min(t.d2, od2));
        if (od1 < t.d1 || (od1 == t.d1 && oj1 < t.j1)) { t.d1 = od1; t.j1 = oj1; }
        t.d2 = nd2;
    }
    return t;
}

__device__ __forceinline__ int dot_s8(const int4 *__restrict__ brow, const int (&qd)[32])
{
    int acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int4 v = __ldg(brow + k);
        acc = __dp4a(v.x, qd[4 * k + 0], acc);
        acc = __dp4a(v.y, qd[4 * k + 1], acc);
        acc = __dp4a(v.z, qd[4 * k + 2], acc);
        acc = __dp4a(v.w, qd[4 * k + 3], acc);
    }
    return acc;
}

// Pair of work item t: the largest k with item_off[k] <= t (item_off has n_pairs + 1 entries).
__device__ __forceinline__ int pair_of_item(const int64_t *__restrict__ item_off, int n_pairs, int64_t t)
{
    int lo = 0, hi = n_pairs;   // invariant: item_off[lo] <= t < item_off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (item_off[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One work item = kQueriesPerItem consecutive queries (in line order) of one pair; one warp per query.
// persistent != 0: the grid is sized to the GPU and blocks take items from a global counter until the batch is
// done (one launch per batch whatever its shape); otherwise block b takes item item_begin + b.
__global__ void __launch_bounds__(kWarpsPerBlock * 32) match_simt_kernel(
    const ImageDev *__restrict__ imgs, const PairDev *__restrict__ pairs, const int64_t *__restrict__ item_off,
    int32_t n_pairs, const int32_t *__restrict__ qorder, int64_t item_begin, int64_t item_end, int32_t persistent,
    int32_t *__restrict__ next, int32_t *__restrict__ match_j, BatchCounters *__restrict__ ctr)
{
    __shared__ int32_t queue[kWarpsPerBlock][64];
    __shared__ unsigned long long bsum[3];
    __shared__ int64_t s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < 3) bsum[threadIdx.x] = 0ull;
    unsigned examined = 0, redecided = 0, cand = 0;
    for (int64_t it = 0;; ++it) {
        __syncthreads();
        if (threadIdx.x == 0) {
            if (persistent) s_item = item_begin + atomicAdd(next, 1);
            else s_item = it == 0 ? item_begin + blockIdx.x : item_end;
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= item_end) break;
        const int pi = pair_of_item(item_off, n_pairs, item);
        const PairDev &P = pairs[pi];
        const ImageDev &A = imgs[P.a];
        const ImageDev &B = imgs[P.b];
        const int k = (int)(item - item_off[pi]) * kWarpsPerBlock + wid;
        if (k >= P.n_a) continue;
        float F[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) F[t] = P.F[t];
        const int s = qorder[P.qoff + k];
        const float2 q = A.xy[s];
        int qd[32];
        {
            const int4 *qrow = reinterpret_cast<const int4 *>(A.desc + (int64_t)s * kDim);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int4 v = __ldg(qrow + t);
                qd[4 * t] = v.x; qd[4 * t + 1] = v.y; qd[4 * t + 2] = v.z; qd[4 * t + 3] = v.w;
            }
        }
        const int qn2 = A.norm[s];
        const BandLine L = band_line(F, q.x, q.y, P.d, (float)B.width, (float)B.height);
        Top2 top{INT_MAX, INT_MAX, INT_MAX};
        int qn = 0;   // queued candidates (warp-uniform)
        unsigned qcand = 0;
        int32_t *wq = queue[wid];
        const int8_t *bdesc = B.desc;
        const int32_t *bnorm = B.norm;
        auto drain = [&](int m) {
            if (lane < m) {
                const int j = wq[lane];
                const int dot = dot_s8(reinterpret_cast<const int4 *>(bdesc + (int64_t)j * kDim), qd);
                top2_push(top, qn2 + bnorm[j] - 2 * dot, j);
            }
        };
        auto visit = [&](bool valid, bool inb, int pos) {
            const unsigned m = __ballot_sync(0xffffffffu, inb);
            if (inb) wq[qn + __popc(m & lanemask_lt())] = pos;
            qn += __popc(m);
            qcand += __popc(m);
            __syncwarp();
            if (qn >= 32) {
                drain(32);
                __syncwarp();
                if (lane < qn - 32) wq[lane] = wq[32 + lane];
                qn -= 32;
                __syncwarp();
            }
        };
        band_walk(B, L, F, q.x, q.y, P.d, visit, examined, redecided);
        drain(qn);
        __syncwarp();
        top = top2_warp_merge(top);
        if (lane == 0) {
            int out = -1;
            if (qcand >= 2 && (int64_t)P.q * P.q * top.d1 < (int64_t)P.p * P.p * top.d2) out = B.perm[top.j1];
            match_j[P.qoff + A.perm[s]] = out;
            cand += qcand;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        examined += __shfl_xor_sync(0xffffffffu, examined, o);
        redecided += __shfl_xor_sync(0xffffffffu, redecided, o);
    }
    if (lane == 0) {
        atomicAdd(&bsum[0], (unsigned long long)cand);
        atomicAdd(&bsum[1], (unsigned long long)examined);
        atomicAdd(&bsum[2], (unsigned long long)redecided);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        BatchCounters *c = ctr + (blockIdx.x % kCounterShards);
        atomicAdd(&c->candidates, bsum[0]);
        atomicAdd(&c->examined, bsum[1]);
        atomicAdd(&c->redecided, bsum[2]);
    }
}

}  // namespace

int match_simt_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, match_simt_kernel, kWarpsPerBlock * 32, 0) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_match_simt(const ImageDev *imgs, const PairDev *pairs, const int64_t *item_off, int32_t n_pairs,
                              const int32_t *qorder, int64_t item_begin, int64_t item_end, int32_t grid,
                              int32_t *next, int32_t *match_j, BatchCounters *ctr, cudaStream_t st)
{
    const int64_t n = item_end - item_begin;
    if (n <= 0) return cudaSuccess;
    const int persistent = grid > 0;
    const int64_t g = persistent ? std::min<int64_t>(grid, n) : n;
    match_simt_kernel<<<(unsigned)g, kWarpsPerBlock * 32, 0, st>>>(imgs, pairs, item_off, n_pairs, qorder, item_begin,
                                                                  item_end, persistent, next, match_j, ctr);
    return cudaGetLastError();
}

}  // namespace gm
