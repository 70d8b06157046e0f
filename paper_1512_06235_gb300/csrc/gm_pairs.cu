// gm_pairs.cu -- gm_select_pairs: candidate image pairs from point-camera co-visibility (Sec. 6.1).
//
// For each query image q, the candidate images are S_q = { i != q : |Points(C_q) & Points(C_i)| > T }, of which the
// top k by co-visible count are kept (ties: the lower image index); the pairs to match are the unique unordered
// pairs {q, i} over all queries, written as rows (a, b, count), a < b, sorted by (a, b).
//
// Three steps on the device:
//   count:  one warp per 3D point adds 1 to the count of every pair of cameras that see it (atomics into the upper
//           triangle of a dense n_cams x n_cams int32 matrix; bit 31 is kept for the selection flag);
//   select: one block per query image finds its top k (a bisection on the count threshold, then the lowest indices
//           among the ties at the threshold) and flags the chosen pairs (atomicOr of bit 31);
//   emit:   per-row counts of flagged pairs, a scan, and one warp per row writing its rows in column order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "gm_ctx.h"

namespace gm {

bool is_device_ptr(const void *p);

namespace {

constexpr int32_t kMaxCams = 16384;
constexpr uint32_t kFlag = 0x80000000u;
constexpr int kSelThreads = 512;

__global__ void covis_count_kernel(const int64_t *__restrict__ point_off, const int32_t *__restrict__ point_cams,
                                   int64_t n_points, int64_t nnz, int32_t n_cams, uint32_t *__restrict__ counts,
                                   unsigned long long *__restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_points; p += warps) {
        const int64_t o = point_off[p], o1 = point_off[p + 1];
        if (o < 0 || o1 < o || o1 > nnz || o1 - o > INT32_MAX) {   // malformed offsets: counted, never read past
            if (lane == 0) atomicAdd(bad, 1ull);
            continue;
        }
        const int d = (int)(o1 - o);
        for (int i = 0; i < d - 1; ++i) {
            const int ci = point_cams[o + i];
            for (int j = i + 1 + lane; j < d; j += 32) {
                const int cj = point_cams[o + j];
                if (ci == cj || (unsigned)ci >= (unsigned)n_cams || (unsigned)cj >= (unsigned)n_cams) {
                    atomicAdd(bad, 1ull);
                    continue;
                }
                const int a = min(ci, cj), b = max(ci, cj);
                atomicAdd(&counts[(int64_t)a * n_cams + b], 1u);
            }
        }
        if (d == 1 && lane == 0 && (unsigned)point_cams[o] >= (unsigned)n_cams) atomicAdd(bad, 1ull);
    }
}

__device__ __forceinline__ uint32_t covis(const uint32_t *counts, int32_t n_cams, int q, int i)
{
    const int a = min(q, i), b = max(q, i);
    return counts[(int64_t)a * n_cams + b] & ~kFlag;
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

// One block per query q: the top k of S_q (count > T) by count, ties to the lower index, flagged in the matrix.
__global__ void __launch_bounds__(kSelThreads) select_kernel(uint32_t *__restrict__ counts, int32_t n_cams,
                                                             int32_t threshold, int32_t top_k)
{
    __shared__ int red[kSelThreads / 32];
    __shared__ int scan_base;
    const int q = blockIdx.x;
    // number of candidates with count >= c (c > threshold), and the largest count
    auto count_ge = [&](uint32_t c) {
        int n = 0;
        for (int i = threadIdx.x; i < n_cams; i += blockDim.x)
            n += (i != q && covis(counts, n_cams, q, i) >= c) ? 1 : 0;
        return block_sum(n, red);
    };
    const uint32_t lo_c = (uint32_t)max(threshold, -1) + 1u;   // counts > T are >= T + 1 (T >= -1)
    const int n_cand = count_ge(lo_c);
    if (n_cand == 0 || top_k <= 0) return;
    uint32_t cstar = lo_c;   // the k-th largest count (all candidates when there are at most k)
    if (n_cand > top_k) {
        uint32_t lo = lo_c, hi = 0x7fffffffu;   // invariant: count_ge(lo) >= top_k, count_ge(hi + 1) < top_k
        int mx = 0;
        for (int i = threadIdx.x; i < n_cams; i += blockDim.x)
            if (i != q) mx = max(mx, (int)covis(counts, n_cams, q, i));
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
        cstar = lo;
    }
    // take every candidate above cstar, and the lowest-index ones at cstar up to k in total
    const int above = n_cand > top_k ? count_ge(cstar + 1) : n_cand;
    const int need_tie = n_cand > top_k ? top_k - above : 0;
    if (threadIdx.x == 0) scan_base = 0;
    __syncthreads();
    for (int base = 0; base < n_cams; base += blockDim.x) {
        const int i = base + threadIdx.x;
        uint32_t c = 0;
        bool take = false, tie = false;
        if (i < n_cams && i != q) {
            c = covis(counts, n_cams, q, i);
            if (n_cand <= top_k) take = c >= lo_c;
            else if (c > cstar) take = true;
            else tie = c == cstar;
        }
        // rank of this tie among the block's ties in index order
        const unsigned bal = __ballot_sync(0xffffffffu, tie);
        const int wrank = __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __popc(bal);
        __syncthreads();
        int before = scan_base;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) before += red[w];
        if (tie && before + wrank < need_tie) take = true;
        if (take) {
            const int a = min(q, i), b = max(q, i);
            atomicOr(&counts[(int64_t)a * n_cams + b], kFlag);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            scan_base += t;
        }
        __syncthreads();
    }
}

// flagged pairs per row a (columns b > a), one warp per row
__global__ void row_count_kernel(const uint32_t *__restrict__ counts, int32_t n_cams, int32_t *__restrict__ rows)
{
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (a >= n_cams) return;
    int n = 0;
    for (int b = a + 1 + lane; b < n_cams; b += 32) n += (counts[(int64_t)a * n_cams + b] & kFlag) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) rows[a] = n;
}

// exclusive scan of the row counts (one block; n_cams <= kMaxCams), off[n_cams] = total
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

__global__ void emit_kernel(const uint32_t *__restrict__ counts, int32_t n_cams, const int64_t *__restrict__ off,
                            int32_t *__restrict__ out)
{
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (a >= n_cams) return;
    int64_t w = off[a];
    for (int b0 = a + 1; b0 < n_cams; b0 += 32) {
        const int b = b0 + lane;
        const uint32_t v = b < n_cams ? counts[(int64_t)a * n_cams + b] : 0u;
        const bool f = (v & kFlag) != 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (f) {
            int32_t *r = out + 3 * (w + __popc(bal & ((1u << lane) - 1u)));
            r[0] = a;
            r[1] = b;
            r[2] = (int32_t)(v & ~kFlag);
        }
        w += __popc(bal);
    }
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
    if (nnz < 0) return fail(GM_ERR_INVALID, "gm_select_pairs: negative point offsets");
    const size_t mat_b = align_up(sizeof(uint32_t) * (size_t)n_cams * n_cams, 256);
    const size_t rows_b = align_up(sizeof(int32_t) * n_cams, 256), off_b = align_up(sizeof(int64_t) * (n_cams + 1), 256);
    const size_t in_b = dev_in ? 0 : align_up(sizeof(int64_t) * (n_points + 1), 256) + align_up(4 * (size_t)nnz + 4, 256);
    gm_status st = ensure_dev(ctx, ctx->d_pairs, mat_b + rows_b + off_b + 256 + in_b);
    if (st != GM_OK) return st;
    char *w = static_cast<char *>(ctx->d_pairs.p);
    uint32_t *counts = reinterpret_cast<uint32_t *>(w);
    int32_t *rows = reinterpret_cast<int32_t *>(w + mat_b);
    int64_t *off = reinterpret_cast<int64_t *>(w + mat_b + rows_b);
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(w + mat_b + rows_b + off_b);
    const int64_t *d_off = point_off;
    const int32_t *d_cams = point_cams;
    if (!dev_in && n_points > 0) {
        char *in = w + mat_b + rows_b + off_b + 256;
        GM_CUDA_P(cudaMemcpyAsync(in, point_off, sizeof(int64_t) * (n_points + 1), cudaMemcpyHostToDevice, s));
        char *cin = in + align_up(sizeof(int64_t) * (n_points + 1), 256);
        GM_CUDA_P(cudaMemcpyAsync(cin, point_cams, 4 * (size_t)nnz, cudaMemcpyHostToDevice, s));
        d_off = reinterpret_cast<const int64_t *>(in);
        d_cams = reinterpret_cast<const int32_t *>(cin);
    }
    GM_CUDA_P(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)n_cams * n_cams, s));
    GM_CUDA_P(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
    if (n_points > 0) {
        const int blocks = std::max(1, std::min<int>((int)((n_points + 7) / 8), ctx->num_sms * 16));
        covis_count_kernel<<<blocks, 256, 0, s>>>(d_off, d_cams, n_points, nnz, n_cams, counts, bad);
        GM_CUDA_P(cudaGetLastError());
    }
    unsigned long long h_bad = 0;
    GM_CUDA_P(cudaMemcpyAsync(&h_bad, bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s));
    GM_CUDA_P(cudaStreamSynchronize(s));
    if (h_bad)
        return fail(GM_ERR_INVALID,
                    "gm_select_pairs: %llu entries repeat a camera within a point, exceed n_cams or have bad offsets",
                    h_bad);
    select_kernel<<<n_cams, kSelThreads, 0, s>>>(counts, n_cams, threshold, top_k);
    GM_CUDA_P(cudaGetLastError());
    row_count_kernel<<<(n_cams * 32 + 255) / 256, 256, 0, s>>>(counts, n_cams, rows);
    row_scan_kernel<<<1, 1024, 0, s>>>(rows, n_cams, off);
    int64_t total = 0;
    GM_CUDA_P(cudaMemcpyAsync(&total, off + n_cams, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GM_CUDA_P(cudaStreamSynchronize(s));
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
        emit_kernel<<<(n_cams * 32 + 255) / 256, 256, 0, s>>>(counts, n_cams, off, dst);
        GM_CUDA_P(cudaGetLastError());
        if (!dev_out) GM_CUDA_P(cudaMemcpyAsync(pairs, dst, sizeof(int32_t) * 3 * (size_t)total, cudaMemcpyDeviceToHost, s));
    }
    GM_CUDA_P(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // extern "C"
