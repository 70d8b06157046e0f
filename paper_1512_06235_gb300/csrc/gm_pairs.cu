// gm_pairs.cu -- gm_select_pairs: candidate image pairs from point-camera co-visibility (Sec. 6.1).
//
// For each query image q, the candidate images are S_q = { i != q : |Points(C_q) & Points(C_i)| > T }, of which the
// top k by co-visible count are kept (ties: the lower image index); the pairs to match are the unique unordered
// pairs {q, i} over all queries, written as rows (a, b, count), a < b, sorted by (a, b).
//
// No n_cams x n_cams matrix: the co-visible counts of one query camera form one row, accumulated in shared memory
// (shared-memory atomics) from the camera's own points.
//   transpose: the point -> cameras lists become camera -> points lists (block-local camera histograms, one global
//              reservation per block and camera, then the block's scatter; the order inside a list is immaterial);
//   select:    one block per query q counts its row, finds its top k (a bisection on the count threshold, then the
//              lowest indices among the ties at the threshold) and keeps only the rule (the k-th count c*_q and the
//              last index taken at c*_q); it also writes the row's sparse part: the cameras b > q with more than T
//              co-visible points, in increasing b, with their counts;
//   count:     one warp per query a walks its sparse row: pair {a, b} is taken iff a chose b or b chose a, which
//              both rules decide from the one symmetric count C[a][b];
//   emit:      the same, writing the taken rows in increasing b at the row's offset (a scan of the counts).
// Work: sum over points of |cameras(p)|^2 shared-memory adds once, reading every camera's point list once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "gm_ctx.h"

namespace gm {

bool is_device_ptr(const void *p);

namespace {

constexpr int32_t kMaxCams = 49152;     // one uint32 row per block: 192 KB of shared memory
constexpr int kRowThreads = 512;
constexpr int kTrThreads = 512;
constexpr int32_t kSmemHistCams = 24576;   // block-local camera histograms in at most 96 KB of shared memory
constexpr int kPairWarps = 8;              // queries per block of the count / emit kernels (one warp each)

struct SelRule {
    uint32_t cstar;    // counts above cstar are taken (0xffffffff: none)
    int32_t tie_last;  // counts equal to cstar are taken for indices <= tie_last (-1: none)
};

// ---- transpose.  Block b takes points [b chunk, (b + 1) chunk).  kSmem: the block's camera histogram lives in shared
// memory (n_cams <= kSmemHistCams) and reaches global memory with one atomic per camera; otherwise every observation
// is a global atomic.  A point with bad offsets or a bad camera entry is counted in *bad and skipped (the same
// entries in both kernels, so that the counts and the scatter agree).
__device__ __forceinline__ bool point_ok(const int64_t *__restrict__ point_off, int64_t p, int64_t nnz, int64_t &o,
                                         int64_t &o1)
{
    o = point_off[p];
    o1 = point_off[p + 1];
    return o >= 0 && o1 >= o && o1 <= nnz;
}

template <bool kSmem>
__global__ void __launch_bounds__(kTrThreads) obs_count_kernel(const int64_t *__restrict__ point_off,
                                                               const int32_t *__restrict__ point_cams, int64_t n_points,
                                                               int64_t nnz, int32_t n_cams, int64_t chunk,
                                                               int32_t *__restrict__ cam_cnt,
                                                               unsigned long long *__restrict__ bad)
{
    extern __shared__ int32_t hist[];
    const int64_t p0 = (int64_t)blockIdx.x * chunk, p1 = min(n_points, p0 + chunk);
    if (kSmem) {
        for (int i = threadIdx.x; i < n_cams; i += blockDim.x) hist[i] = 0;
        __syncthreads();
    }
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        int64_t o, o1;
        if (!point_ok(point_off, p, nnz, o, o1)) {
            atomicAdd(bad, 1ull);
            continue;
        }
        for (int64_t j = o; j < o1; ++j) {
            const int c = point_cams[j];
            if ((unsigned)c >= (unsigned)n_cams) atomicAdd(bad, 1ull);
            else atomicAdd(kSmem ? &hist[c] : &cam_cnt[c], 1);
        }
    }
    if (kSmem) {
        __syncthreads();
        for (int i = threadIdx.x; i < n_cams; i += blockDim.x)
            if (hist[i]) atomicAdd(&cam_cnt[i], hist[i]);
    }
}

template <bool kSmem>
__global__ void __launch_bounds__(kTrThreads) obs_fill_kernel(const int64_t *__restrict__ point_off,
                                                              const int32_t *__restrict__ point_cams, int64_t n_points,
                                                              int64_t nnz, int32_t n_cams, int64_t chunk,
                                                              const int32_t *__restrict__ cam_off,
                                                              int32_t *__restrict__ cursor, int32_t *__restrict__ cam_pts)
{
    extern __shared__ int32_t hist[];
    const int64_t p0 = (int64_t)blockIdx.x * chunk, p1 = min(n_points, p0 + chunk);
    if (kSmem) {   // the block's counts, then its range in every camera list, then the scatter
        for (int i = threadIdx.x; i < n_cams; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            int64_t o, o1;
            if (!point_ok(point_off, p, nnz, o, o1)) continue;
            for (int64_t j = o; j < o1; ++j) {
                const int c = point_cams[j];
                if ((unsigned)c < (unsigned)n_cams) atomicAdd(&hist[c], 1);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n_cams; i += blockDim.x)
            if (hist[i]) hist[i] = cam_off[i] + atomicAdd(&cursor[i], hist[i]);
        __syncthreads();
    }
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        int64_t o, o1;
        if (!point_ok(point_off, p, nnz, o, o1)) continue;
        for (int64_t j = o; j < o1; ++j) {
            const int c = point_cams[j];
            if ((unsigned)c >= (unsigned)n_cams) continue;
            const int at = kSmem ? atomicAdd(&hist[c], 1) : cam_off[c] + atomicAdd(&cursor[c], 1);
            cam_pts[at] = (int32_t)p;
        }
    }
}

__device__ __forceinline__ int block_sum(int v, int *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

__device__ __forceinline__ bool taken(const SelRule &r, uint32_t c, int i)
{
    return c > r.cstar || (c == r.cstar && i <= r.tie_last);
}

// The co-visible counts of camera q with every camera, in shared memory (row[q] = 0): one thread per point of q,
// four points' dependent loads (point id, offsets, camera list) in flight per thread.  Every point of q must list q
// exactly once (else *bad); a camera listed twice by one point is caught by that camera's own row.
__device__ void count_row(uint32_t *row, int q, int32_t n_cams, const int32_t *__restrict__ cam_off,
                          const int32_t *__restrict__ cam_pts, const int64_t *__restrict__ point_off,
                          const int32_t *__restrict__ point_cams, unsigned long long *bad)
{
    for (int i = threadIdx.x; i < n_cams; i += blockDim.x) row[i] = 0u;
    __syncthreads();
    constexpr int kU = 4;
    const int k0 = cam_off[q], k1 = cam_off[q + 1];
    for (int k = k0 + (int)threadIdx.x; k < k1; k += kU * (int)blockDim.x) {
        int32_t p[kU];
        int64_t o[kU], e[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int kk = k + u * (int)blockDim.x;
            p[u] = kk < k1 ? __ldg(cam_pts + kk) : -1;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            o[u] = p[u] >= 0 ? __ldg(point_off + p[u]) : 0;
            e[u] = p[u] >= 0 ? __ldg(point_off + p[u] + 1) : 0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            int own = 0;
            for (int64_t j = o[u]; j < e[u]; ++j) {
                const int c = __ldg(point_cams + j);
                if (c == q) ++own;
                else if ((unsigned)c < (unsigned)n_cams) atomicAdd(&row[c], 1u);
            }
            if (p[u] >= 0 && own != 1) atomicAdd(bad, 1ull);
        }
    }
    __syncthreads();
}

// One block per query q: its selection rule, and its sparse row (cameras b > q with a count above T, increasing b)
// in the pool at an atomically reserved offset (rows that do not fit are counted in *pool_used all the same: the
// caller grows the pool to that total and runs the selection again).
__global__ void __launch_bounds__(kRowThreads) select_kernel(
    int32_t n_cams, const int32_t *__restrict__ cam_off, const int32_t *__restrict__ cam_pts,
    const int64_t *__restrict__ point_off, const int32_t *__restrict__ point_cams, int32_t threshold, int32_t top_k,
    SelRule *__restrict__ rules, uint2 *__restrict__ pool, unsigned long long pool_cap,
    unsigned long long *__restrict__ pool_used, unsigned long long *__restrict__ row_ptr, int32_t *__restrict__ row_len,
    unsigned long long *__restrict__ bad)
{
    extern __shared__ uint32_t row[];
    __shared__ int red[kRowThreads / 32];
    __shared__ int scan_base;
    __shared__ unsigned long long row_base;
    const int q = blockIdx.x;
    count_row(row, q, n_cams, cam_off, cam_pts, point_off, point_cams, bad);
    const uint32_t lo_c = (uint32_t)(threshold + 1);   // counts > T are >= T + 1 (T >= -1)
    {
        auto count_ge = [&](uint32_t c) {
            int n = 0;
            for (int i = threadIdx.x; i < n_cams; i += blockDim.x) n += (i != q && row[i] >= c) ? 1 : 0;
            return block_sum(n, red);
        };
        const int n_cand = count_ge(lo_c);
        SelRule r{0xffffffffu, -1};
        if (n_cand > 0 && top_k > 0) {
            if (n_cand <= top_k) {
                r.cstar = lo_c - 1u;   // every candidate: counts above T (T = -1: all, cstar wraps to 0xffffffff)
                if (threshold < 0) { r.cstar = 0u; r.tie_last = n_cams; }
            } else {
                uint32_t lo = lo_c, hi = 0;   // invariant: count_ge(lo) >= top_k, count_ge(hi + 1) < top_k
                int mx = 0;
                for (int i = threadIdx.x; i < n_cams; i += blockDim.x)
                    if (i != q) mx = max(mx, (int)row[i]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                __syncthreads();
                if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
                __syncthreads();
                mx = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
                hi = (uint32_t)mx;
                while (lo < hi) {
                    const uint32_t mid = lo + (hi - lo + 1) / 2;
                    if (count_ge(mid) >= top_k) lo = mid;
                    else hi = mid - 1;
                }
                const uint32_t cstar = lo;
                const int need_tie = top_k - count_ge(cstar + 1);   // >= 1
                // the need_tie-th camera (in index order) whose count equals cstar
                __syncthreads();
                if (threadIdx.x == 0) scan_base = 0;
                __shared__ int tie_last;
                if (threadIdx.x == 0) tie_last = -1;
                __syncthreads();
                for (int base = 0; base < n_cams; base += blockDim.x) {
                    const int i = base + threadIdx.x;
                    const bool tie = i < n_cams && i != q && row[i] == cstar;
                    const unsigned bal = __ballot_sync(0xffffffffu, tie);
                    const int wrank = __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
                    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __popc(bal);
                    __syncthreads();
                    int before = scan_base;
                    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) before += red[w];
                    if (tie && before + wrank == need_tie - 1) tie_last = i;
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        int t = 0;
                        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
                        scan_base += t;
                    }
                    __syncthreads();
                }
                r.cstar = cstar;
                r.tie_last = tie_last;
            }
        }
        if (threadIdx.x == 0) rules[q] = r;
    }
    // the sparse row
    int n = 0;
    for (int b = q + 1 + (int)threadIdx.x; b < n_cams; b += blockDim.x) n += row[b] >= lo_c ? 1 : 0;
    n = block_sum(n, red);
    if (threadIdx.x == 0) {
        row_base = n ? atomicAdd(pool_used, (unsigned long long)n) : 0ull;
        row_ptr[q] = row_base;
        row_len[q] = row_base + (unsigned long long)n <= pool_cap ? n : 0;   // a row that does not fit reads as empty
        scan_base = 0;
    }
    __syncthreads();
    if (n == 0 || row_base + (unsigned long long)n > pool_cap) return;
    for (int base = q + 1; base < n_cams; base += blockDim.x) {
        const int b = base + threadIdx.x;
        const bool t = b < n_cams && row[b] >= lo_c;
        const unsigned bal = __ballot_sync(0xffffffffu, t);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __popc(bal);
        __syncthreads();
        if (t) {
            int before = scan_base;
            for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) before += red[w];
            pool[row_base + before + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = make_uint2((uint32_t)b, row[b]);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t2 = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t2 += red[w];
            scan_base += t2;
        }
        __syncthreads();
    }
}

// One warp per query a: pairs {a, b}, b > a, from a's sparse row, taken by a's rule or by b's (the count is
// symmetric).  kWrite = false: rows[a] = how many; true: write them at off[a], in increasing b.
template <bool kWrite>
__global__ void __launch_bounds__(kPairWarps * 32) pair_kernel(int32_t n_cams, const SelRule *__restrict__ rules,
                                                              const uint2 *__restrict__ pool,
                                                              const unsigned long long *__restrict__ row_ptr,
                                                              const int32_t *__restrict__ row_len,
                                                              int32_t *__restrict__ rows,
                                                              const int64_t *__restrict__ off, int32_t *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * kPairWarps + (threadIdx.x >> 5);
    if (q >= n_cams) return;
    const SelRule rq = rules[q];
    const int len = row_len[q];
    const uint2 *e = pool + row_ptr[q];
    const int64_t w0 = kWrite ? off[q] : 0;
    int run = 0;
    for (int i0 = 0; i0 < len; i0 += 32) {
        const int i = i0 + lane;
        bool t = false;
        uint2 v = make_uint2(0u, 0u);
        if (i < len) {
            v = e[i];
            t = taken(rq, v.y, (int)v.x) || taken(rules[v.x], v.y, q);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, t);
        if (kWrite && t) {
            int32_t *o = out + 3 * (w0 + run + __popc(bal & ((1u << lane) - 1u)));
            o[0] = q;
            o[1] = (int32_t)v.x;
            o[2] = (int32_t)v.y;
        }
        run += __popc(bal);
    }
    if (!kWrite && lane == 0) rows[q] = run;
}

// exclusive scan of the row counts (one block), off[n_cams] = total
__global__ void __launch_bounds__(1024) row_scan_kernel(const int32_t *__restrict__ rows, int32_t n_cams,
                                                        int64_t *__restrict__ off)
{
    __shared__ int64_t part[1024];
    const int per = (n_cams + 1023) / 1024;
    const int s0 = threadIdx.x * per, s1 = min(n_cams, s0 + per);
    int64_t t = 0;
    for (int i = s0; i < s1; ++i) t += rows[i];
    part[threadIdx.x] = t;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int i = s0; i < s1; ++i) {
        off[i] = run;
        run += rows[i];
    }
    if (threadIdx.x == 1023) off[n_cams] = part[1023];
}

#define GM_CUDA_P(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return gm::fail(GM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace
}  // namespace gm

extern "C" {

gm_status gm_select_pairs(gm_ctx *ctx, int32_t n_cams, int64_t n_points, const int64_t *point_off,
                          const int32_t *point_cams, int32_t threshold, int32_t top_k, int32_t *pairs, int64_t cap,
                          int64_t *n_written)
{
    gm::NvtxRange nvtx_("gm_select_pairs");
    using namespace gm;
    if (!ctx || n_cams < 0 || n_cams > kMaxCams || n_points < 0 || (n_points > 0 && (!point_off || !point_cams)) ||
        threshold < -1 || top_k < 0 || cap < 0 || (cap > 0 && !pairs) || !n_written)
        return fail(GM_ERR_INVALID, "gm_select_pairs: bad arguments (n_cams must be in [0, %d], T >= -1, k >= 0)",
                    kMaxCams);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA_P(cudaSetDevice(ctx->device));
    *n_written = 0;
    if (n_cams == 0) return GM_OK;
    cudaStream_t s = ctx->ws.stream;
    // inputs on the device
    const bool dev_in = n_points == 0 || is_device_ptr(point_off);
    if (n_points > 0 && dev_in != is_device_ptr(point_cams))
        return fail(GM_ERR_INVALID, "gm_select_pairs: point_off and point_cams must both be host or both device");
    int64_t nnz = 0;
    if (n_points > 0) {
        if (dev_in) {
            GM_CUDA_P(cudaMemcpyAsync(&nnz, point_off + n_points, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            GM_CUDA_P(cudaStreamSynchronize(s));
        } else {
            nnz = point_off[n_points];
        }
    }
    if (nnz < 0 || nnz > INT32_MAX - 1 || n_points > INT32_MAX - 1)
        return fail(GM_ERR_INVALID, "gm_select_pairs: negative point offsets or more than 2^31 observations");
    const size_t cnt_b = align_up(sizeof(int32_t) * (n_cams + 1), 256);   // counts, then offsets (scan), cursors
    const size_t bs_b = align_up(sizeof(int32_t) * (n_cams / 1024 + 2), 256);
    const size_t pts_b = align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1), 256);
    const size_t rule_b = align_up(sizeof(SelRule) * n_cams, 256), rows_b = align_up(sizeof(int32_t) * n_cams, 256);
    const size_t off_b = align_up(sizeof(int64_t) * (n_cams + 1), 256);
    const size_t rp_b = align_up(sizeof(unsigned long long) * n_cams, 256);
    const size_t in_b = dev_in ? 0 : align_up(sizeof(int64_t) * (n_points + 1), 256) + align_up(4 * (size_t)nnz + 4, 256);
    gm_status st =
        ensure_dev(ctx, ctx->d_pairs, 3 * cnt_b + bs_b + pts_b + rule_b + 2 * rows_b + off_b + rp_b + 256 + in_b);
    if (st != GM_OK) return st;
    char *w = static_cast<char *>(ctx->d_pairs.p);
    int32_t *cam_cnt = reinterpret_cast<int32_t *>(w);
    int32_t *cam_off = reinterpret_cast<int32_t *>(w + cnt_b);
    int32_t *cursor = reinterpret_cast<int32_t *>(w + 2 * cnt_b);
    w += 3 * cnt_b;
    int32_t *bsum = reinterpret_cast<int32_t *>(w);
    int32_t *cam_pts = reinterpret_cast<int32_t *>(w + bs_b);
    w += bs_b + pts_b;
    SelRule *rules = reinterpret_cast<SelRule *>(w);
    int32_t *rows = reinterpret_cast<int32_t *>(w + rule_b);
    int32_t *row_len = reinterpret_cast<int32_t *>(w + rule_b + rows_b);
    w += rule_b + 2 * rows_b;
    int64_t *off = reinterpret_cast<int64_t *>(w);
    unsigned long long *row_ptr = reinterpret_cast<unsigned long long *>(w + off_b);
    // bad[0]: entries outside [0, n_cams) or bad offsets; bad[1]: points listing a camera twice; bad[2]: pool use
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(w + off_b + rp_b);
    const int64_t *d_off = point_off;
    const int32_t *d_cams = point_cams;
    if (!dev_in && n_points > 0) {
        char *in = reinterpret_cast<char *>(bad) + 256;
        GM_CUDA_P(cudaMemcpyAsync(in, point_off, sizeof(int64_t) * (n_points + 1), cudaMemcpyHostToDevice, s));
        char *cin = in + align_up(sizeof(int64_t) * (n_points + 1), 256);
        GM_CUDA_P(cudaMemcpyAsync(cin, point_cams, 4 * (size_t)nnz, cudaMemcpyHostToDevice, s));
        d_off = reinterpret_cast<const int64_t *>(in);
        d_cams = reinterpret_cast<const int32_t *>(cin);
    }
    static const cudaError_t attr = [] {
        cudaError_t e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(uint32_t) * kMaxCams));
        for (const void *f : {(const void *)obs_count_kernel<true>, (const void *)obs_fill_kernel<true>})
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(int32_t) * kSmemHistCams));
        return e;
    }();
    GM_CUDA_P(attr);
    GM_CUDA_P(cudaMemsetAsync(cam_cnt, 0, sizeof(int32_t) * (n_cams + 1), s));
    GM_CUDA_P(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (n_cams + 1), s));
    GM_CUDA_P(cudaMemsetAsync(bad, 0, 3 * sizeof(unsigned long long), s));
    // transpose: every block a contiguous range of points (a few thousand observations each)
    const int64_t tr_grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * 2, (n_points + 1023) / 1024));
    const int64_t chunk = (n_points + tr_grid - 1) / tr_grid;
    const bool smem_hist = n_cams <= kSmemHistCams;
    const size_t tr_smem = smem_hist ? sizeof(int32_t) * (size_t)n_cams : 0;
    if (n_points > 0) {
        if (smem_hist)
            obs_count_kernel<true><<<(unsigned)tr_grid, kTrThreads, tr_smem, s>>>(d_off, d_cams, n_points, nnz, n_cams,
                                                                               chunk, cam_cnt, bad);
        else
            obs_count_kernel<false><<<(unsigned)tr_grid, kTrThreads, 0, s>>>(d_off, d_cams, n_points, nnz, n_cams, chunk,
                                                                              cam_cnt, bad);
        GM_CUDA_P(cudaGetLastError());
    }
    GM_CUDA_P(launch_exclusive_scan(cam_cnt, n_cams, cam_off, bsum, s));
    if (n_points > 0) {
        if (smem_hist)
            obs_fill_kernel<true><<<(unsigned)tr_grid, kTrThreads, tr_smem, s>>>(d_off, d_cams, n_points, nnz, n_cams,
                                                                              chunk, cam_off, cursor, cam_pts);
        else
            obs_fill_kernel<false><<<(unsigned)tr_grid, kTrThreads, 0, s>>>(d_off, d_cams, n_points, nnz, n_cams, chunk,
                                                                             cam_off, cursor, cam_pts);
        GM_CUDA_P(cudaGetLastError());
    }
    // selection and the sparse rows (the pool grows to what a first run needed, then the selection runs again),
    // then the taken pairs per query
    const size_t row_smem = sizeof(uint32_t) * (size_t)n_cams;
    unsigned long long pool_cap =
        std::max<unsigned long long>(ctx->d_pairs_pool.bytes / sizeof(uint2), std::max(65536ull, 16ull * n_cams));
    int64_t total = 0;
    unsigned long long h_bad[3] = {0, 0, 0};
    for (int attempt = 0; attempt < 2; ++attempt) {
        if ((st = ensure_dev(ctx, ctx->d_pairs_pool, sizeof(uint2) * (size_t)pool_cap)) != GM_OK) return st;
        uint2 *pool = static_cast<uint2 *>(ctx->d_pairs_pool.p);
        GM_CUDA_P(cudaMemsetAsync(bad + 1, 0, 2 * sizeof(unsigned long long), s));
        select_kernel<<<n_cams, kRowThreads, row_smem, s>>>(n_cams, cam_off, cam_pts, d_off, d_cams, threshold, top_k,
                                                            rules, pool, pool_cap, bad + 2, row_ptr, row_len, bad + 1);
        pair_kernel<false><<<(n_cams + kPairWarps - 1) / kPairWarps, kPairWarps * 32, 0, s>>>(
            n_cams, rules, pool, row_ptr, row_len, rows, off, nullptr);
        row_scan_kernel<<<1, 1024, 0, s>>>(rows, n_cams, off);
        GM_CUDA_P(cudaGetLastError());
        GM_CUDA_P(cudaMemcpyAsync(&total, off + n_cams, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GM_CUDA_P(cudaMemcpyAsync(h_bad, bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s));
        GM_CUDA_P(cudaStreamSynchronize(s));
        if (h_bad[0])
            return fail(GM_ERR_INVALID, "gm_select_pairs: %llu entries exceed n_cams or have bad offsets", h_bad[0]);
        if (h_bad[1])
            return fail(GM_ERR_INVALID, "gm_select_pairs: %llu points list one camera more than once", h_bad[1]);
        if (h_bad[2] <= pool_cap) break;
        if (attempt == 1) return fail(GM_ERR_CUDA, "gm_select_pairs: sparse rows grew between two identical runs");
        pool_cap = h_bad[2];
    }
    *n_written = total;
    if (total > cap)
        return fail(GM_ERR_NOMEM, "gm_select_pairs: %lld pairs exceed cap %lld", (long long)total, (long long)cap);
    if (total > 0) {
        int32_t *dst = pairs;
        const bool dev_out = is_device_ptr(pairs);
        if (!dev_out) {
            if ((st = ensure_dev(ctx, ctx->d_pairs_out, sizeof(int32_t) * 3 * (size_t)total)) != GM_OK) return st;
            dst = static_cast<int32_t *>(ctx->d_pairs_out.p);
        }
        pair_kernel<true><<<(n_cams + kPairWarps - 1) / kPairWarps, kPairWarps * 32, 0, s>>>(
            n_cams, rules, static_cast<const uint2 *>(ctx->d_pairs_pool.p), row_ptr, row_len, rows, off, dst);
        GM_CUDA_P(cudaGetLastError());
        if (!dev_out) GM_CUDA_P(cudaMemcpyAsync(pairs, dst, sizeof(int32_t) * 3 * (size_t)total, cudaMemcpyDeviceToHost, s));
    }
    GM_CUDA_P(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // extern "C"
