// gm_bucket.cu -- grid bucketing of images (App. A Step 1: cell index per feature, sort by cell, prefix scan of the
// cell counts gives each cell's start).  Done once per image; the result stays resident.  Every launch covers all
// images of a registration batch (each thread finds its image in a prefix table).
//
// A counting sort: histogram (atomics) -> exclusive scan (block-parallel, two passes, over the count arrays of all
// images at once; each image's offsets are its segment minus the segment start) -> scatter (one thread per
// keypoint, atomic cursor per cell).  The order inside a cell is whatever the atomics give: no result depends on
// it (every band decision is per keypoint, and an accepted match has a unique nearest neighbour because ties are
// rejected).  Two layouts are built: column-major (cells of a grid column contiguous) and row-major.  Descriptors
// are then copied in column-major order, recentred to int8 (b - 128, the bit pattern b ^ 0x80), with their
// squared norms, an fp16 copy and the point records of the tensor-core path.
#include <cuda_fp16.h>

#include <cstdint>

#include "gm_internal.h"

namespace gm {
namespace {

// Column-major and row-major cell index of a keypoint; a keypoint outside [0,W) x [0,H) (or NaN) goes to the
// extra cell gx*gy at the end of both layouts, so every launch stays in bounds; the host rejects such images.
__device__ __forceinline__ bool cell_of(float2 p, float W, float H, float inv_cs, int gx, int gy, int &ccol,
                                        int &crow)
{
    if (!(p.x >= 0.0f && p.x < W && p.y >= 0.0f && p.y < H)) {
        ccol = crow = gx * gy;
        return false;
    }
    const int cx = min((int)floorf(p.x * inv_cs), gx - 1);   // cs is a power of two: p.x * inv_cs is exact
    const int cy = min((int)floorf(p.y * inv_cs), gy - 1);
    ccol = cx * gy + cy;
    crow = cy * gx + cx;
    return true;
}

constexpr int kScanBlock = 1024;

__device__ __forceinline__ int block_incl_scan(int v, int32_t *wsum, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, s);
        if (lane >= s) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, s);
            if (lane >= s) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    total = wsum[nw - 1];
    return (wid > 0 ? wsum[wid - 1] : 0) + incl;
}

// Pass 1: per block of kScanBlock counts, the local exclusive scan into off[] and the block total.
__global__ void __launch_bounds__(kScanBlock) scan_local_kernel(const int32_t *__restrict__ cnt, int32_t m,
                                                                 int32_t *__restrict__ off, int32_t *__restrict__ bsum)
{
    __shared__ int32_t wsum[32];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const int v = i < m ? cnt[i] : 0;
    int total;
    const int incl = block_incl_scan(v, wsum, total);
    if (i < m) off[i] = incl - v;
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Pass 2: add the totals of the earlier blocks; the last block also writes off[m] (the grand total).
__global__ void __launch_bounds__(kScanBlock) scan_add_kernel(const int32_t *__restrict__ bsum, int32_t nblocks,
                                                               int32_t m, int32_t *__restrict__ off)
{
    __shared__ int32_t wsum[32];
    __shared__ int32_t base;
    int acc = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += blockDim.x) acc += bsum[k];
    int total;
    block_incl_scan(acc, wsum, total);
    if (threadIdx.x == 0) base = total;
    __syncthreads();
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < m) off[i] += base;
    if (blockIdx.x == nblocks - 1 && threadIdx.x == 0) off[m] = base + bsum[blockIdx.x];
}

cudaError_t exclusive_scan_impl(const int32_t *cnt, int32_t m, int32_t *off, int32_t *bsum, cudaStream_t st)
{
    const int nb = (m + kScanBlock - 1) / kScanBlock;
    scan_local_kernel<<<nb, kScanBlock, 0, st>>>(cnt, m, off, bsum);
    scan_add_kernel<<<nb, kScanBlock, 0, st>>>(bsum, nb, m, off);
    return cudaGetLastError();
}

__device__ __forceinline__ int find_job(const int64_t *__restrict__ prefix, int K, int64_t g)
{
    int lo = 0, hi = K;   // largest k with prefix[k] <= g
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void batch_count_kernel(const BucketJob *__restrict__ jobs, const int64_t *__restrict__ kp_prefix, int K,
                                   int64_t n_total, int32_t *work, unsigned long long *bad)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_total) return;
    const int k = find_job(kp_prefix, K, g);
    const BucketJob &J = jobs[k];
    int ccol, crow;
    if (!cell_of(J.xy_raw[g - J.kp_base], (float)J.width, (float)J.height, 1.0f / (float)(1 << J.cell_shift), J.gx,
                 J.gy, ccol, crow))
        atomicAdd(&bad[k], 1ull);
    int32_t *cnt = work + J.cnt_base;
    atomicAdd(&cnt[ccol], 1);
    atomicAdd(&cnt[J.m + 1 + crow], 1);
}

// scan holds the exclusive scan of the whole work array; each image's offsets are its segment minus the
// segment's first value, written to the image's col_off / row_off and (for the cells) back into work as cursors.
__global__ void batch_offsets_kernel(const BucketJob *__restrict__ jobs, const int64_t *__restrict__ cnt_prefix,
                                     int K, int64_t S, const int32_t *__restrict__ scan, int32_t *work)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S) return;
    const int k = find_job(cnt_prefix, K, p);
    const BucketJob &J = jobs[k];
    const int64_t q = p - J.cnt_base;
    const bool row = q > J.m;
    const int c = (int)(row ? q - (J.m + 1) : q);
    const int64_t seg = J.cnt_base + (row ? J.m + 1 : 0);
    const int32_t v = scan[p] - scan[seg];
    (row ? J.row_off : J.col_off)[c] = v;
    if (c < J.m) work[p] = v;
}

__global__ void batch_scatter_kernel(const BucketJob *__restrict__ jobs, const int64_t *__restrict__ kp_prefix, int K,
                                     int64_t n_total, int32_t *work, bool row_pass)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_total) return;
    const int k = find_job(kp_prefix, K, g);
    const BucketJob &J = jobs[k];
    const int i = (int)(g - J.kp_base);
    const float2 p = J.xy_raw[i];
    int ccol, crow;
    cell_of(p, (float)J.width, (float)J.height, 1.0f / (float)(1 << J.cell_shift), J.gx, J.gy, ccol, crow);
    int32_t *cur = work + J.cnt_base;
    if (!row_pass) {
        const int pos = atomicAdd(&cur[ccol], 1);
        J.perm[pos] = i;
        J.xy[pos] = p;
        J.inv_perm[i] = pos;
    } else {
        const int pos = atomicAdd(&cur[J.m + 1 + crow], 1);
        J.xy_r[pos] = p;
        J.idx_r[pos] = J.inv_perm[i];
    }
}

// Descriptors in cell order: eight lanes per keypoint, 16 bytes each (a warp moves four rows per load, so that
// more bytes are in flight when the rows are read from page-locked host memory), recentred int8, fp16 and the norms.
// The input rows are read in their own order (sequential reads over the host link when they are read in place) and
// written to their cell-order positions (inv_perm, from the scatter before).
__global__ void batch_desc_kernel(const BucketJob *__restrict__ jobs, const int64_t *__restrict__ kp_prefix, int K,
                                  int64_t n_total)
{
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int part = threadIdx.x & 7;
    const bool live = g < n_total;   // every lane takes part in the shuffles below
    int sq = 0;
    const BucketJob *J = nullptr;
    int row = 0;
    if (live) {
        const int k = find_job(kp_prefix, K, g);
        J = &jobs[k];
        const int src = (int)(g - J->kp_base);
        row = J->inv_perm[src];
        uint4 w = reinterpret_cast<const uint4 *>(J->desc_raw + (int64_t)src * kDim)[part];
        w.x ^= 0x80808080u; w.y ^= 0x80808080u; w.z ^= 0x80808080u; w.w ^= 0x80808080u;
        reinterpret_cast<uint4 *>(J->desc + (int64_t)row * kDim)[part] = w;
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        uint32_t h[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int t = 0; t < 4; t += 2) {
                const int v0 = (int)(int8_t)((ws[q] >> (8 * t)) & 0xffu);
                const int v1 = (int)(int8_t)((ws[q] >> (8 * t + 8)) & 0xffu);
                sq += v0 * v0 + v1 * v1;
                h[2 * q + t / 2] = (uint32_t)__half_as_ushort(__int2half_rn(v0)) |
                                   ((uint32_t)__half_as_ushort(__int2half_rn(v1)) << 16);
            }
        }
        uint4 *dh = reinterpret_cast<uint4 *>(J->desc_h + (int64_t)row * kDim) + 2 * part;
        dh[0] = make_uint4(h[0], h[1], h[2], h[3]);
        dh[1] = make_uint4(h[4], h[5], h[6], h[7]);
    }
#pragma unroll
    for (int s = 4; s > 0; s >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s);
    if (live && part == 0) {
        J->norm[row] = sq;
        J->norm256[row] = sq * 256;
        // the norm row of the whole-image matcher: -(sq >> 11), -(sq & 2047) / 2, 1024 (all exact in fp16)
        const uint32_t h0 = (uint32_t)__half_as_ushort(__float2half_rn(-(float)(sq >> 11))) |
                            ((uint32_t)__half_as_ushort(__float2half_rn(-0.5f * (float)(sq & 2047))) << 16);
        const uint32_t h1 = (uint32_t)__half_as_ushort(__float2half_rn(1024.0f));
        uint4 *dx = reinterpret_cast<uint4 *>(J->ext_h + (int64_t)row * 16);
        dx[0] = make_uint4(h0, h1, 0u, 0u);
        dx[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// records of every image plus one sentinel each: index g over sum (n + 1), image k owns [kp_base + k, ...]
__global__ void batch_records_kernel(const BucketJob *__restrict__ jobs, const int64_t *__restrict__ rec_prefix,
                                     int K, int64_t n_rec)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_rec) return;
    const int k = find_job(rec_prefix, K, g);
    const BucketJob &J = jobs[k];
    const int i = (int)(g - (J.kp_base + k));
    if (i == J.n) {
        const int nan = 0x7fc00000;
        J.rec[i] = make_int4(nan, nan, 0, 0);
        return;
    }
    const float2 p = J.xy[i];
    J.rec[i] = make_int4(__float_as_int(p.x), __float_as_int(p.y), J.norm256[i], i);
}

unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

cudaError_t exclusive_scan(const int32_t *cnt, int32_t m, int32_t *off, int32_t *bsum, cudaStream_t st)
{
    return exclusive_scan_impl(cnt, m, off, bsum, st);
}

}  // namespace

cudaError_t launch_exclusive_scan(const int32_t *cnt, int32_t m, int32_t *off, int32_t *bsum, cudaStream_t st)
{
    return exclusive_scan_impl(cnt, m, off, bsum, st);
}

cudaError_t launch_bucket_batch_count(const BucketJob *jobs, const int64_t *kp_prefix, int32_t K, int64_t n_total,
                                      int32_t *work, int64_t S, unsigned long long *bad, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int32_t) * (size_t)S, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long) * (size_t)K, st);
    if (e != cudaSuccess) return e;
    if (n_total > 0) batch_count_kernel<<<blocks_for(n_total, 256), 256, 0, st>>>(jobs, kp_prefix, K, n_total, work, bad);
    return cudaGetLastError();
}

cudaError_t launch_bucket_batch_build(const BucketJob *jobs, const int64_t *kp_prefix, const int64_t *cnt_prefix,
                                      const int64_t *rec_prefix, int32_t K, int64_t n_total, int32_t *work, int64_t S,
                                      int32_t *scan, int32_t *bsum, cudaStream_t st)
{
    if (S > INT32_MAX - 1) return cudaErrorInvalidValue;
    cudaError_t e = exclusive_scan(work, (int32_t)S, scan, bsum, st);
    if (e != cudaSuccess) return e;
    batch_offsets_kernel<<<blocks_for(S, 256), 256, 0, st>>>(jobs, cnt_prefix, K, S, scan, work);
    if (n_total > 0) {
        batch_scatter_kernel<<<blocks_for(n_total, 256), 256, 0, st>>>(jobs, kp_prefix, K, n_total, work, false);
        batch_scatter_kernel<<<blocks_for(n_total, 256), 256, 0, st>>>(jobs, kp_prefix, K, n_total, work, true);
        batch_desc_kernel<<<blocks_for(n_total * 8, 256), 256, 0, st>>>(jobs, kp_prefix, K, n_total);
    }
    // the record index space has one extra entry (the sentinel) per image: rec_prefix[k] = kp_prefix[k] + k
    batch_records_kernel<<<blocks_for(n_total + K, 256), 256, 0, st>>>(jobs, rec_prefix, K, n_total + K);
    return cudaGetLastError();
}

}  // namespace gm
