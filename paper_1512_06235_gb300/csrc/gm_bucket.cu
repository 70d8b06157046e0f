// gm_bucket.cu -- grid bucketing of one image (App. A Step 1: cell index per feature, sort by cell, prefix scan
// of the cell counts gives each cell's start).  Done once per image; the result stays resident.
//
// A counting sort: histogram (atomics) -> exclusive scan (block-parallel, two passes) -> scatter (one thread per
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

__global__ void bucket_count_kernel(const float2 *__restrict__ xy, int32_t n, float W, float H, float inv_cs,
                                    int gx, int gy, int32_t *cnt_col, int32_t *cnt_row,
                                    unsigned long long *bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int ccol, crow;
    if (!cell_of(xy[i], W, H, inv_cs, gx, gy, ccol, crow)) atomicAdd(bad, 1ull);
    atomicAdd(&cnt_col[ccol], 1);
    atomicAdd(&cnt_row[crow], 1);
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

cudaError_t exclusive_scan(const int32_t *cnt, int32_t m, int32_t *off, int32_t *bsum, cudaStream_t st)
{
    const int nb = (m + kScanBlock - 1) / kScanBlock;
    scan_local_kernel<<<nb, kScanBlock, 0, st>>>(cnt, m, off, bsum);
    scan_add_kernel<<<nb, kScanBlock, 0, st>>>(bsum, nb, m, off);
    return cudaGetLastError();
}

// Column-major scatter: one thread per keypoint (cur: per-cell cursors, initialised to the offsets).
__global__ void scatter_col_kernel(const float2 *__restrict__ xy_raw, int32_t n, float W, float H, float inv_cs,
                                   int gx, int gy, int32_t *__restrict__ cur, float2 *__restrict__ xy,
                                   int32_t *__restrict__ perm, int32_t *__restrict__ inv_perm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 p = xy_raw[i];
    int ccol, crow;
    cell_of(p, W, H, inv_cs, gx, gy, ccol, crow);
    const int pos = atomicAdd(&cur[ccol], 1);
    perm[pos] = i;
    xy[pos] = p;
    inv_perm[i] = pos;
}

// Row-major scatter (after the column-major one: idx_r holds column-major positions).
__global__ void scatter_row_kernel(const float2 *__restrict__ xy_raw, int32_t n, float W, float H, float inv_cs,
                                   int gx, int gy, int32_t *__restrict__ cur, const int32_t *__restrict__ inv_perm,
                                   float2 *__restrict__ xy_r, int32_t *__restrict__ idx_r)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 p = xy_raw[i];
    int ccol, crow;
    cell_of(p, W, H, inv_cs, gx, gy, ccol, crow);
    const int pos = atomicAdd(&cur[crow], 1);
    xy_r[pos] = p;
    idx_r[pos] = inv_perm[i];
}

// One warp per sorted row: recentred int8 copy, squared norm and fp16 copy of the descriptor.
__global__ void desc_permute_kernel(const uint8_t *__restrict__ desc_raw, const int32_t *__restrict__ perm,
                                    int32_t n, int8_t *__restrict__ desc, int32_t *__restrict__ norm,
                                    int32_t *__restrict__ norm256, uint16_t *__restrict__ desc_h)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int src = perm[warp];
    const uint32_t w = reinterpret_cast<const uint32_t *>(desc_raw + (int64_t)src * kDim)[lane] ^ 0x80808080u;
    reinterpret_cast<uint32_t *>(desc + (int64_t)warp * kDim)[lane] = w;
    int sq = 0;
    uint32_t h01 = 0, h23 = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int v = (int)(int8_t)((w >> (8 * k)) & 0xffu);
        sq += v * v;
        const uint16_t hb = __half_as_ushort(__int2half_rn(v));
        if (k < 2) h01 |= (uint32_t)hb << (16 * k);
        else h23 |= (uint32_t)hb << (16 * (k - 2));
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s);
    if (lane == 0) {
        norm[warp] = sq;
        norm256[warp] = sq * 256;
    }
    if (desc_h) reinterpret_cast<uint2 *>(desc_h + (int64_t)warp * kDim)[lane] = make_uint2(h01, h23);
}

// Point records for the tensor-core path: (x, y, |b'|^2 * 256, column-major position) in column-major order,
// followed by a sentinel whose NaN coordinates fail every band test.
__global__ void records_kernel(const float2 *__restrict__ xy, const int32_t *__restrict__ norm256, int32_t n,
                               int4 *__restrict__ rec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) {
        const int nan = 0x7fc00000;
        rec[n] = make_int4(nan, nan, 0, 0);
        return;
    }
    const float2 p = xy[i];
    rec[i] = make_int4(__float_as_int(p.x), __float_as_int(p.y), norm256[i], i);
}

}  // namespace

cudaError_t launch_bucket_count(const float2 *xy_raw, int32_t n, int32_t width, int32_t height, int32_t cell_shift,
                                int32_t gx, int32_t gy, int32_t *work, unsigned long long *bad, cudaStream_t st)
{
    // work: two count arrays of gx*gy + 2 entries (the cells, the out-of-image cell, a spare)
    const int m = gx * gy + 1;
    const float inv_cs = 1.0f / (float)(1 << cell_shift);
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int32_t) * 2 * (m + 1), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if (n > 0)
        bucket_count_kernel<<<(n + 255) / 256, 256, 0, st>>>(xy_raw, n, (float)width, (float)height, inv_cs, gx, gy,
                                                             work, work + (m + 1), bad);
    return cudaGetLastError();
}

cudaError_t launch_bucket_build(const float2 *xy_raw, const uint8_t *desc_raw, int32_t n, int32_t width,
                                int32_t height, int32_t cell_shift, int32_t gx, int32_t gy, float2 *xy, int32_t *perm,
                                int32_t *inv_perm, int8_t *desc, int32_t *norm, int32_t *norm256, int32_t *col_off,
                                float2 *xy_r, int32_t *idx_r, int32_t *row_off, uint16_t *desc_h, int4 *rec,
                                int32_t *work, cudaStream_t st)
{
    // col_off / row_off hold gx*gy + 2 entries: the cells, the out-of-image cell, the total
    const int m = gx * gy + 1;
    const float inv_cs = 1.0f / (float)(1 << cell_shift);
    int32_t *cnt_col = work, *cnt_row = work + (m + 1), *bsum = work + 2 * (m + 1);
    cudaError_t e;
    if ((e = exclusive_scan(cnt_col, m, col_off, bsum, st)) != cudaSuccess) return e;
    if ((e = exclusive_scan(cnt_row, m, row_off, bsum + (m + kScanBlock - 1) / kScanBlock, st)) != cudaSuccess)
        return e;
    // cursors start at the offsets (reuse the count arrays)
    if ((e = cudaMemcpyAsync(cnt_col, col_off, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(cnt_row, row_off, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    if (n > 0) {
        const int nb = (n + 255) / 256;
        scatter_col_kernel<<<nb, 256, 0, st>>>(xy_raw, n, (float)width, (float)height, inv_cs, gx, gy, cnt_col, xy,
                                               perm, inv_perm);
        scatter_row_kernel<<<nb, 256, 0, st>>>(xy_raw, n, (float)width, (float)height, inv_cs, gx, gy, cnt_row,
                                               inv_perm, xy_r, idx_r);
        desc_permute_kernel<<<(n + 7) / 8, 256, 0, st>>>(desc_raw, perm, n, desc, norm, norm256, desc_h);
    }
    records_kernel<<<(n + 1 + 255) / 256, 256, 0, st>>>(xy, norm256, n, rec);
    return cudaGetLastError();
}

}  // namespace gm
