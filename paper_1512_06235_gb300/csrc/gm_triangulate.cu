// gm_triangulate.cu -- gm_triangulate: linear least-squares triangulation of feature tracks (Sec. 6.2, end).
//
// Nodes are numbered image-major over the caller's image list (node = first node of image k + feature index) and
// labelled by their component (gm_merge_tracks).  Every component with at least two nodes is a track; tracks are
// numbered in increasing order of their root (smallest node).  Each observation -- camera P (3 x 4) of its image
// and the feature's coordinates (x, y) -- contributes the rows x P3 - P1 and y P3 - P2 to A = [A3 | a4]; the point
// solves the normal equations (A3^T A3) X = -A3^T a4 (FP64; a singular system gives NaN).
//   sizes:   component sizes (atomics);
//   number:  flags of the roots of tracks, scanned into track numbers;
//   accum:   one thread per node adds its two rows to its track's six distinct entries of A3^T A3 and three of
//            -A3^T a4 (FP64 atomics; the order of the additions varies from run to run in the last bits);
//   solve:   one thread per track, Cramer's rule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "gm_ctx.h"

namespace gm {
namespace {

struct TriImage {
    const float2 *xy;          // cell order
    const int32_t *inv_perm;   // caller's feature index -> cell position
    int64_t base;              // first node
    int32_t n;
    int32_t pad_;
};

__global__ void tri_sizes_kernel(const int64_t *__restrict__ labels, int64_t n_nodes, int32_t *__restrict__ size,
                                 unsigned long long *bad)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_nodes; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = labels[v];
        if (r < 0 || r > v || labels[r] != r) {   // a label is the smallest node of its component, its own label
            atomicAdd(bad, 1ull);
            continue;
        }
        atomicAdd(&size[r], 1);
    }
}

__global__ void tri_flags_kernel(const int64_t *__restrict__ labels, const int32_t *__restrict__ size, int64_t n_nodes,
                                 int32_t *__restrict__ flag)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_nodes; v += (int64_t)gridDim.x * blockDim.x)
        flag[v] = (labels[v] == v && size[v] >= 2) ? 1 : 0;
}

__device__ __forceinline__ int find_image(const TriImage *__restrict__ imgs, int n_images, int64_t v)
{
    int lo = 0, hi = n_images;   // largest k with base[k] <= v
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (imgs[mid].base <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void tri_accum_kernel(const int64_t *__restrict__ labels, const int32_t *__restrict__ size,
                                 const int32_t *__restrict__ track_of, int64_t n_nodes,
                                 const TriImage *__restrict__ imgs, int n_images, const double *__restrict__ P,
                                 double *__restrict__ acc, int64_t *__restrict__ roots, int32_t *__restrict__ n_views)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_nodes; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = labels[v];
        if (r < 0 || r > v || size[r] < 2) continue;
        const int32_t t = track_of[r];
        const int k = find_image(imgs, n_images, v);
        const TriImage &I = imgs[k];
        const int f = (int)(v - I.base);
        const float2 p = I.xy[I.inv_perm[f]];
        const double x = (double)p.x, y = (double)p.y;
        const double *Pk = P + 12 * (int64_t)k;
        double r1[4], r2[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            r1[c] = x * Pk[8 + c] - Pk[c];
            r2[c] = y * Pk[8 + c] - Pk[4 + c];
        }
        double *a = acc + 9 * (int64_t)t;   // M00 M01 M02 M11 M12 M22, b0 b1 b2
        atomicAdd(&a[0], r1[0] * r1[0] + r2[0] * r2[0]);
        atomicAdd(&a[1], r1[0] * r1[1] + r2[0] * r2[1]);
        atomicAdd(&a[2], r1[0] * r1[2] + r2[0] * r2[2]);
        atomicAdd(&a[3], r1[1] * r1[1] + r2[1] * r2[1]);
        atomicAdd(&a[4], r1[1] * r1[2] + r2[1] * r2[2]);
        atomicAdd(&a[5], r1[2] * r1[2] + r2[2] * r2[2]);
        atomicAdd(&a[6], -(r1[0] * r1[3] + r2[0] * r2[3]));
        atomicAdd(&a[7], -(r1[1] * r1[3] + r2[1] * r2[3]));
        atomicAdd(&a[8], -(r1[2] * r1[3] + r2[2] * r2[3]));
        if (r == v) {
            roots[t] = r;
            n_views[t] = size[r];
        }
    }
}

__global__ void tri_solve_kernel(const double *__restrict__ acc, int64_t n_tracks, double *__restrict__ X)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tracks; t += (int64_t)gridDim.x * blockDim.x) {
        const double *a = acc + 9 * t;
        const double m00 = a[0], m01 = a[1], m02 = a[2], m11 = a[3], m12 = a[4], m22 = a[5];
        const double b0 = a[6], b1 = a[7], b2 = a[8];
        const double c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
        const double det = m00 * c00 + m01 * c01 + m02 * c02;
        double *o = X + 3 * t;
        if (det == 0.0 || !isfinite(det)) {
            o[0] = o[1] = o[2] = nan("");
            continue;
        }
        const double c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
        const double id = 1.0 / det;
        o[0] = (c00 * b0 + c01 * b1 + c02 * b2) * id;
        o[1] = (c01 * b0 + c11 * b1 + c12 * b2) * id;
        o[2] = (c02 * b0 + c12 * b1 + c22 * b2) * id;
    }
}

#define GM_CUDA_R(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return gm::fail(GM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace
}  // namespace gm

extern "C" {

gm_status gm_triangulate(gm_ctx *ctx, int32_t n_images, const int32_t *image_ids, const double *P, int64_t n_nodes,
                         const int64_t *labels, int64_t cap, double *X, int64_t *roots, int32_t *n_views,
                         int64_t *n_tracks)
{
    gm::NvtxRange nvtx_("gm_triangulate");
    using namespace gm;
    if (!ctx || n_images < 0 || (n_images > 0 && (!image_ids || !P)) || n_nodes < 0 || (n_nodes > 0 && !labels) ||
        cap < 0 || (cap > 0 && (!X || !roots || !n_views)) || !n_tracks)
        return fail(GM_ERR_INVALID, "gm_triangulate: bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA_R(cudaSetDevice(ctx->device));
    *n_tracks = 0;
    // the node numbering of the caller's image list
    std::vector<TriImage> imgs(n_images);
    int64_t total = 0;
    for (int32_t k = 0; k < n_images; ++k) {
        auto it = ctx->images.find(image_ids[k]);
        if (image_ids[k] < 0 || it == ctx->images.end())
            return fail(GM_ERR_NOT_FOUND, "gm_triangulate: image %d not registered", image_ids[k]);
        const ImageDev &d = it->second->dev;
        imgs[k] = TriImage{d.xy, d.inv_perm, total, d.n, 0};
        total += d.n;
    }
    if (total != n_nodes)
        return fail(GM_ERR_INVALID, "gm_triangulate: n_nodes %lld differs from the images' %lld features",
                    (long long)n_nodes, (long long)total);
    if (n_nodes == 0) return GM_OK;
    if (n_nodes > INT32_MAX - 1) return fail(GM_ERR_INVALID, "gm_triangulate: too many nodes");
    cudaStream_t s = ctx->ws.stream;
    const bool dev_l = is_device_ptr(labels), dev_p = is_device_ptr(P);
    const size_t N = (size_t)n_nodes;
    const size_t img_b = align_up(sizeof(TriImage) * std::max(n_images, 1), 256);
    const size_t p_b = align_up(sizeof(double) * 12 * std::max(n_images, 1), 256);
    const size_t lab_b = dev_l ? 0 : align_up(8 * N, 256);
    const size_t sz_b = align_up(4 * N, 256), fl_b = align_up(4 * N, 256), tr_b = align_up(4 * (N + 1), 256);
    const size_t bs_b = align_up(4 * (N / 1024 + 2), 256);
    gm_status st = ensure_dev(ctx, ctx->d_tri, img_b + p_b + lab_b + sz_b + fl_b + tr_b + bs_b + 256);
    if (st != GM_OK) return st;
    char *w = static_cast<char *>(ctx->d_tri.p);
    TriImage *d_imgs = reinterpret_cast<TriImage *>(w);
    double *d_P = reinterpret_cast<double *>(w + img_b);
    const int64_t *d_lab = labels;
    char *q = w + img_b + p_b;
    if (!dev_l) {
        GM_CUDA_R(cudaMemcpyAsync(q, labels, 8 * N, cudaMemcpyHostToDevice, s));
        d_lab = reinterpret_cast<const int64_t *>(q);
        q += lab_b;
    }
    int32_t *size = reinterpret_cast<int32_t *>(q);
    int32_t *flag = reinterpret_cast<int32_t *>(q + sz_b);
    int32_t *track_of = reinterpret_cast<int32_t *>(q + sz_b + fl_b);
    int32_t *bsum = reinterpret_cast<int32_t *>(q + sz_b + fl_b + tr_b);
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(q + sz_b + fl_b + tr_b + bs_b);
    GM_CUDA_R(cudaMemcpyAsync(d_imgs, imgs.data(), sizeof(TriImage) * n_images, cudaMemcpyHostToDevice, s));
    GM_CUDA_R(cudaMemcpyAsync(d_P, P, sizeof(double) * 12 * n_images,
                              dev_p ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    GM_CUDA_R(cudaMemsetAsync(size, 0, 4 * N, s));
    GM_CUDA_R(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
    const int grid = std::max(1, ctx->num_sms * 8);
    tri_sizes_kernel<<<grid, 256, 0, s>>>(d_lab, n_nodes, size, bad);
    tri_flags_kernel<<<grid, 256, 0, s>>>(d_lab, size, n_nodes, flag);
    GM_CUDA_R(launch_exclusive_scan(flag, (int32_t)n_nodes, track_of, bsum, s));
    int32_t nt = 0;
    unsigned long long h_bad = 0;
    GM_CUDA_R(cudaMemcpyAsync(&nt, track_of + n_nodes, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GM_CUDA_R(cudaMemcpyAsync(&h_bad, bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s));
    GM_CUDA_R(cudaStreamSynchronize(s));
    if (h_bad)
        return fail(GM_ERR_INVALID, "gm_triangulate: %llu labels are not the smallest node of a component", h_bad);
    *n_tracks = nt;
    if (nt > cap) return fail(GM_ERR_NOMEM, "gm_triangulate: %d tracks exceed cap %lld", nt, (long long)cap);
    if (nt == 0) return GM_OK;
    // per-track accumulators and outputs (device; copied out when the caller's buffers are host memory)
    const bool dev_o = is_device_ptr(X);
    if (is_device_ptr(roots) != dev_o || is_device_ptr(n_views) != dev_o)
        return fail(GM_ERR_INVALID, "gm_triangulate: X, roots and n_views must all be host or all device memory");
    const size_t acc_b = align_up(sizeof(double) * 9 * nt, 256), x_b = align_up(sizeof(double) * 3 * nt, 256);
    const size_t r_b = align_up(sizeof(int64_t) * nt, 256), v_b = align_up(sizeof(int32_t) * nt, 256);
    if ((st = ensure_dev(ctx, ctx->d_tri_out, acc_b + (dev_o ? 0 : x_b + r_b + v_b))) != GM_OK) return st;
    char *o = static_cast<char *>(ctx->d_tri_out.p);
    double *acc = reinterpret_cast<double *>(o);
    double *dX = dev_o ? X : reinterpret_cast<double *>(o + acc_b);
    int64_t *dR = dev_o ? roots : reinterpret_cast<int64_t *>(o + acc_b + x_b);
    int32_t *dV = dev_o ? n_views : reinterpret_cast<int32_t *>(o + acc_b + x_b + r_b);
    GM_CUDA_R(cudaMemsetAsync(acc, 0, sizeof(double) * 9 * nt, s));
    tri_accum_kernel<<<grid, 256, 0, s>>>(d_lab, size, track_of, n_nodes, d_imgs, n_images, d_P, acc, dR, dV);
    tri_solve_kernel<<<std::max(1, std::min(grid, (nt + 255) / 256)), 256, 0, s>>>(acc, nt, dX);
    GM_CUDA_R(cudaGetLastError());
    if (!dev_o) {
        GM_CUDA_R(cudaMemcpyAsync(X, dX, sizeof(double) * 3 * nt, cudaMemcpyDeviceToHost, s));
        GM_CUDA_R(cudaMemcpyAsync(roots, dR, sizeof(int64_t) * nt, cudaMemcpyDeviceToHost, s));
        GM_CUDA_R(cudaMemcpyAsync(n_views, dV, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost, s));
    }
    GM_CUDA_R(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // extern "C"
