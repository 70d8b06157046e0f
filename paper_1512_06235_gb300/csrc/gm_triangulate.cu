// gm_triangulate.cu -- linear least-squares triangulation of feature tracks (Sec. 6.3).
//
// gm_triangulate: the merged tracks (connected components of all matches, gm_merge_tracks).
// gm_triangulate_image_tracks: the per-image tracks that Sec. 6.3 triangulates before merging -- every query
// image's features with their matches in all its candidate images.
//
// Nodes are numbered image-major over the caller's image list (node = first node of image k + feature index) and
// labelled by their component (gm_merge_tracks).  Every component with at least two nodes is a track; tracks are
// numbered in increasing order of their root (smallest node).  Each observation -- camera P (3 x 4) of its image
// and the feature's coordinates (x, y) -- contributes the rows x P3 - P1 and y P3 - P2 to A = [A3 | a4]; the point
// solves the normal equations (A3^T A3) X = -A3^T a4 (FP64; a singular system gives NaN).
//   sizes:   component sizes (atomics);
//   number:  flags of the roots of tracks, scanned into track numbers;
//   accum:   every node of a track adds its two rows to its track's six distinct entries of A3^T A3 and three of
//            -A3^T a4, a warp's track nodes 32 at a time (FP64 atomics; the order of the additions varies from run
//            to run in the last bits);
//   solve:   one thread per track, Cramer's rule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <unordered_map>
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

// One observation (node v of track t = track_of[r], r its root) into its track's sums.
__device__ __forceinline__ void tri_accum_one(int64_t v, const int64_t *__restrict__ labels,
                                              const int32_t *__restrict__ size, const int32_t *__restrict__ track_of,
                                              const TriImage *__restrict__ imgs, int n_images,
                                              const double *__restrict__ P, double *__restrict__ acc,
                                              int64_t *__restrict__ roots, int32_t *__restrict__ n_views)
{
    const int64_t r = labels[v];
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

constexpr int kAccumThreads = 256;

// Every node of a track adds its observation.  The FP64 pipe bounds this pass (it runs at a small fraction of the
// FP32 rate on GB300), and many nodes belong to no track, so each warp queues its nodes that do in shared memory
// and adds them 32 at a time: every FP64 instruction runs on a full warp (the last round of each warp excepted).
__global__ void __launch_bounds__(kAccumThreads)
    tri_accum_kernel(const int64_t *__restrict__ labels, const int32_t *__restrict__ size,
                     const int32_t *__restrict__ track_of, int64_t n_nodes, const TriImage *__restrict__ imgs,
                     int n_images, const double *__restrict__ P, double *__restrict__ acc,
                     int64_t *__restrict__ roots, int32_t *__restrict__ n_views)
{
    __shared__ int64_t queue[kAccumThreads / 32][64];
    const int lane = threadIdx.x & 31;
    int64_t *q = queue[threadIdx.x >> 5];
    int n = 0;   // queued nodes (the same in every lane)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_nodes; base += stride) {
        const int64_t v = base + lane;
        bool obs = false;
        if (v < n_nodes) {
            const int64_t r = labels[v];
            obs = r >= 0 && r <= v && size[r] >= 2;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, obs);
        if (obs) q[n + __popc(bal & ((1u << lane) - 1u))] = v;
        n += __popc(bal);
        __syncwarp();
        if (n >= 32) {
            tri_accum_one(q[lane], labels, size, track_of, imgs, n_images, P, acc, roots, n_views);
            __syncwarp();
            if (lane < n - 32) q[lane] = q[lane + 32];
            n -= 32;
            __syncwarp();
        }
    }
    if (lane < n) tri_accum_one(q[lane], labels, size, track_of, imgs, n_images, P, acc, roots, n_views);
}

// Cramer's rule on the normal equations a = (M00 M01 M02 M11 M12 M22, b0 b1 b2); NaN if singular.
__device__ __forceinline__ void tri_solve(const double *a, double *o)
{
    const double m00 = a[0], m01 = a[1], m02 = a[2], m11 = a[3], m12 = a[4], m22 = a[5];
    const double b0 = a[6], b1 = a[7], b2 = a[8];
    const double c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
    const double det = m00 * c00 + m01 * c01 + m02 * c02;
    if (det == 0.0 || !isfinite(det)) {
        o[0] = o[1] = o[2] = nan("");
        return;
    }
    const double c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
    const double id = 1.0 / det;
    o[0] = (c00 * b0 + c01 * b1 + c02 * b2) * id;
    o[1] = (c01 * b0 + c11 * b1 + c12 * b2) * id;
    o[2] = (c02 * b0 + c12 * b1 + c22 * b2) * id;
}

__global__ void tri_solve_kernel(const double *__restrict__ acc, int64_t n_tracks, double *__restrict__ X)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tracks; t += (int64_t)gridDim.x * blockDim.x)
        tri_solve(acc + 9 * t, X + 3 * t);
}

// Adds the observation (x, y) of camera Pk (3 x 4, row-major) to the normal equations a: the rows x P3 - P1 and
// y P3 - P2 of A = [A3 | a4] into A3^T A3 (six distinct entries) and -A3^T a4.
__device__ __forceinline__ void tri_add(double *a, const double *__restrict__ Pk, double x, double y)
{
    double r1[4], r2[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        r1[c] = x * Pk[8 + c] - Pk[c];
        r2[c] = y * Pk[8 + c] - Pk[4 + c];
    }
    a[0] += r1[0] * r1[0] + r2[0] * r2[0];
    a[1] += r1[0] * r1[1] + r2[0] * r2[1];
    a[2] += r1[0] * r1[2] + r2[0] * r2[2];
    a[3] += r1[1] * r1[1] + r2[1] * r2[1];
    a[4] += r1[1] * r1[2] + r2[1] * r2[2];
    a[5] += r1[2] * r1[2] + r2[2] * r2[2];
    a[6] -= r1[0] * r1[3] + r2[0] * r2[3];
    a[7] -= r1[1] * r1[3] + r2[1] * r2[3];
    a[8] -= r1[2] * r1[3] + r2[2] * r2[3];
}

// ---- per-image tracks
// Pairs of the caller's list: pair p's rows are matches[off[p] .. off[p+1]), image indices ka (query), kb.
struct TrkPair {
    int32_t ka, kb;
};

// Row m of the match list belongs to pair p with off[p] <= m < off[p+1] (largest such p).
__device__ __forceinline__ int pair_of_row(const int64_t *__restrict__ off, int n_pairs, int64_t m)
{
    int lo = 0, hi = n_pairs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= m) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Every row names features inside its images, and i increases strictly within a pair (one match per query); each
// valid row is entered in its pair's dense query index: slot[pbase[p] + i] = row (slots start at -1).
__global__ void trk_scatter_kernel(const int2 *__restrict__ rows, int64_t n_rows, const int64_t *__restrict__ off,
                                   int n_pairs, const TrkPair *__restrict__ pairs, const TriImage *__restrict__ imgs,
                                   const int64_t *__restrict__ pbase, int32_t *__restrict__ slot,
                                   unsigned long long *bad)
{
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n_rows; m += (int64_t)gridDim.x * blockDim.x) {
        const int p = pair_of_row(off, n_pairs, m);
        const int2 r = rows[m];
        bool ok = r.x >= 0 && r.x < imgs[pairs[p].ka].n && r.y >= 0 && r.y < imgs[pairs[p].kb].n;
        if (m + 1 < off[p + 1]) ok = ok && rows[m + 1].x > r.x;
        if (!ok) atomicAdd(bad, 1ull);
        else slot[pbase[p] + r.x] = (int32_t)m;
    }
}

// Pass 1: per node v, the number of pairs of its image in which it matched, cnt[v], and flag[v] = (cnt[v] > 0).
// Consecutive nodes read consecutive entries of each pair's dense query index.
__global__ void trk_count_kernel(int64_t n_nodes, const TriImage *__restrict__ imgs, int n_images,
                                 const int32_t *__restrict__ img_poff, const int32_t *__restrict__ img_pairs,
                                 const int64_t *__restrict__ pbase, const int32_t *__restrict__ slot,
                                 int32_t *__restrict__ flag, int32_t *__restrict__ cnt)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_nodes; v += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_image(imgs, n_images, v);
        const int f = (int)(v - imgs[k].base);
        int c = 0;
        for (int t = img_poff[k]; t < img_poff[k + 1]; ++t) c += __ldg(slot + pbase[img_pairs[t]] + f) >= 0;
        flag[v] = c > 0;
        cnt[v] = c;
    }
}

// Pass 2: the node of every track, nodes[track_of[v]] = v for each flagged node v.
__global__ void trk_list_kernel(int64_t n_nodes, const int32_t *__restrict__ track_of, int64_t *__restrict__ nodes)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_nodes; v += (int64_t)gridDim.x * blockDim.x)
        if (track_of[v + 1] != track_of[v]) nodes[track_of[v]] = v;
}

constexpr int kSolveThreads = 256;
constexpr int kCntBins = 64;   // match counts from kCntBins - 1 up share the last bin

// Pass 3: the normal equations of every track -- its node's own observation, then one per pair of its image (in
// the caller's order) in which the node matched -- solved into X[t].  The FP64 pipe bounds this pass (it runs at a
// small fraction of the FP32 rate on GB300), so its work runs in rounds: in each round every lane walks its
// image's pairs (integer loads only) to its next match, then the warp adds one observation per lane together.  A
// warp takes as many rounds as its longest track has matches; each block first orders its 256 tracks by match
// count (a counting sort in shared memory), so a warp's tracks have nearly equal counts.  Which lane takes a track
// changes nothing in its result: each track adds its observations in its own order, deterministically.
__global__ void __launch_bounds__(kSolveThreads)
    trk_solve_kernel(int32_t n_tracks, const int64_t *__restrict__ nodes, const int32_t *__restrict__ cnt,
                     const TriImage *__restrict__ imgs, int n_images, const int32_t *__restrict__ img_poff,
                     const int32_t *__restrict__ img_pairs, const TrkPair *__restrict__ pairs,
                     const int64_t *__restrict__ pbase, const int32_t *__restrict__ slot,
                     const int2 *__restrict__ rows, const double *__restrict__ P, double *__restrict__ X,
                     int32_t *__restrict__ n_views)
{
    __shared__ int bin_off[kCntBins];
    __shared__ int64_t s_node[kSolveThreads];
    __shared__ int32_t s_cnt[kSolveThreads], s_track[kSolveThreads];
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < kCntBins) bin_off[tid] = 0;
    __syncthreads();
    const int64_t t_in = (int64_t)blockIdx.x * kSolveThreads + tid;
    int64_t v_in = 0;
    int c_in = 0;
    if (t_in < n_tracks) {
        v_in = nodes[t_in];
        c_in = cnt[v_in];
    }
    const int bin = min(c_in, kCntBins - 1);
    atomicAdd(&bin_off[bin], 1);
    __syncthreads();
    if (tid < 32) {   // exclusive scan of the 64 bins, two per lane
        const int h0 = bin_off[2 * lane], h1 = bin_off[2 * lane + 1];
        int x = h0 + h1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        bin_off[2 * lane] = x - h0 - h1;
        bin_off[2 * lane + 1] = x - h1;
    }
    __syncthreads();
    const int pos = atomicAdd(&bin_off[bin], 1);
    s_node[pos] = v_in;
    s_cnt[pos] = t_in < n_tracks ? c_in : 0;
    s_track[pos] = t_in < n_tracks ? tid : -1;
    __syncthreads();
    const int64_t v = s_node[tid];
    const int need = s_cnt[tid];
    const bool live = s_track[tid] >= 0;
    const int64_t t = (int64_t)blockIdx.x * kSolveThreads + s_track[tid];
    double a[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int f = 0, pt = 0, pe = 0;
    if (live) {
        const int k = find_image(imgs, n_images, v);
        const TriImage &Q = imgs[k];
        f = (int)(v - Q.base);
        const float2 q = Q.xy[Q.inv_perm[f]];
        tri_add(a, P + 12 * (int64_t)k, (double)q.x, (double)q.y);
        pt = img_poff[k];
        pe = img_poff[k + 1];
    }
    const int rounds = __reduce_max_sync(0xffffffffu, need);
    for (int r = 0; r < rounds; ++r) {
        int32_t m = -1;
        int p = 0;
        if (r < need) {
            while (pt < pe) {
                p = img_pairs[pt++];
                m = __ldg(slot + pbase[p] + f);
                if (m >= 0) break;
            }
        }
        if (m >= 0) {
            const int kb = pairs[p].kb;
            const TriImage &B = imgs[kb];
            const float2 b = B.xy[B.inv_perm[__ldg(&rows[m].y)]];
            tri_add(a, P + 12 * (int64_t)kb, (double)b.x, (double)b.y);
        }
    }
    if (live) {
        tri_solve(a, X + 3 * t);
        n_views[t] = 1 + need;
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
    // four blocks per SM: each warp then sees enough nodes that most of its rounds are full
    tri_accum_kernel<<<std::max(1, ctx->num_sms * 4), kAccumThreads, 0, s>>>(d_lab, size, track_of, n_nodes, d_imgs,
                                                                            n_images, d_P, acc, dR, dV);
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

gm_status gm_triangulate_image_tracks(gm_ctx *ctx, int32_t n_images, const int32_t *image_ids, const double *P,
                                      int32_t n_pairs, const int32_t *pair_images, const int64_t *pair_off,
                                      const int32_t *matches, int64_t cap, double *X, int64_t *nodes,
                                      int32_t *n_views, int64_t *n_tracks)
{
    gm::NvtxRange nvtx_("gm_triangulate_image_tracks");
    using namespace gm;
    if (!ctx || n_images < 0 || (n_images > 0 && (!image_ids || !P)) || n_pairs < 0 ||
        (n_pairs > 0 && (!pair_images || !pair_off)) || cap < 0 || (cap > 0 && (!X || !nodes || !n_views)) ||
        !n_tracks)
        return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA_R(cudaSetDevice(ctx->device));
    *n_tracks = 0;
    std::vector<TriImage> imgs(n_images);
    std::unordered_map<int32_t, int32_t> index;
    int64_t total = 0;
    for (int32_t k = 0; k < n_images; ++k) {
        auto it = ctx->images.find(image_ids[k]);
        if (image_ids[k] < 0 || it == ctx->images.end())
            return fail(GM_ERR_NOT_FOUND, "gm_triangulate_image_tracks: image %d not registered", image_ids[k]);
        if (!index.emplace(image_ids[k], k).second)
            return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: image %d listed twice", image_ids[k]);
        const ImageDev &d = it->second->dev;
        imgs[k] = TriImage{d.xy, d.inv_perm, total, d.n, 0};
        total += d.n;
    }
    if (total > INT32_MAX - 1) return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: too many nodes");
    // the pairs: image indices, offsets on the host (validated), and every image's pairs as the query side
    std::vector<int64_t> off(n_pairs + 1, 0);
    cudaStream_t s = ctx->ws.stream;
    if (n_pairs > 0) {
        GM_CUDA_R(cudaMemcpyAsync(off.data(), pair_off, sizeof(int64_t) * (n_pairs + 1), cudaMemcpyDefault, s));
        GM_CUDA_R(cudaStreamSynchronize(s));
    }
    if (off[0] != 0) return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: pair_off[0] must be 0");
    std::vector<TrkPair> pairs(n_pairs);
    std::vector<int64_t> keys(n_pairs);
    std::vector<int32_t> img_poff(n_images + 1, 0), img_pairs(n_pairs);
    for (int32_t p = 0; p < n_pairs; ++p) {
        auto ia = index.find(pair_images[2 * p]), ib = index.find(pair_images[2 * p + 1]);
        if (ia == index.end() || ib == index.end())
            return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: pair %d names an image outside image_ids", p);
        if (ia->second == ib->second)
            return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: pair %d matches an image with itself", p);
        if (off[p + 1] < off[p])
            return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: pair_off decreases at pair %d", p);
        pairs[p] = TrkPair{ia->second, ib->second};
        keys[p] = (int64_t)ia->second * n_images + ib->second;
        ++img_poff[ia->second + 1];
    }
    std::vector<int64_t> sorted_keys(keys);
    std::sort(sorted_keys.begin(), sorted_keys.end());
    if (std::adjacent_find(sorted_keys.begin(), sorted_keys.end()) != sorted_keys.end())
        return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: an ordered pair is listed twice");
    for (int32_t k = 0; k < n_images; ++k) img_poff[k + 1] += img_poff[k];
    {
        std::vector<int32_t> fill(img_poff.begin(), img_poff.end() - 1);
        for (int32_t p = 0; p < n_pairs; ++p) img_pairs[fill[pairs[p].ka]++] = p;   // the caller's order
    }
    const int64_t M = off[n_pairs];
    if (M > 0 && !matches) return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: null matches");
    if (total == 0 || M == 0) return GM_OK;
    const bool dev_m = is_device_ptr(matches), dev_p = is_device_ptr(P);
    const size_t N = (size_t)total;
    const size_t img_b = align_up(sizeof(TriImage) * std::max(n_images, 1), 256);
    const size_t p_b = align_up(sizeof(double) * 12 * std::max(n_images, 1), 256);
    const size_t off_b = align_up(sizeof(int64_t) * (n_pairs + 1), 256);
    const size_t pr_b = align_up(sizeof(TrkPair) * std::max(n_pairs, 1), 256);
    const size_t ip_b = align_up(sizeof(int32_t) * (n_images + 1), 256);
    const size_t il_b = align_up(sizeof(int32_t) * std::max(n_pairs, 1), 256);
    const size_t m_b = dev_m ? 0 : align_up(sizeof(int32_t) * 2 * (size_t)M, 256);
    const size_t fl_b = align_up(4 * N, 256), tr_b = align_up(4 * (N + 1), 256);
    const size_t bs_b = align_up(4 * (N / 1024 + 2), 256);
    // every pair's dense query index: one int32 per feature of its query image
    std::vector<int64_t> pbase(n_pairs + 1, 0);
    for (int32_t p = 0; p < n_pairs; ++p) pbase[p + 1] = pbase[p] + imgs[pairs[p].ka].n;
    const size_t pb_b = align_up(sizeof(int64_t) * (n_pairs + 1), 256);
    const size_t sl_b = align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(pbase[n_pairs], 1), 256);
    gm_status st = ensure_dev(ctx, ctx->d_tri, img_b + p_b + off_b + pr_b + ip_b + il_b + m_b + fl_b + tr_b + bs_b +
                                                   256 + pb_b + sl_b + fl_b);
    if (st != GM_OK) return st;
    char *w = static_cast<char *>(ctx->d_tri.p);
    TriImage *d_imgs = reinterpret_cast<TriImage *>(w);
    w += img_b;
    double *d_P = reinterpret_cast<double *>(w);
    w += p_b;
    int64_t *d_off = reinterpret_cast<int64_t *>(w);
    w += off_b;
    TrkPair *d_pairs = reinterpret_cast<TrkPair *>(w);
    w += pr_b;
    int32_t *d_ipoff = reinterpret_cast<int32_t *>(w);
    w += ip_b;
    int32_t *d_ipairs = reinterpret_cast<int32_t *>(w);
    w += il_b;
    const int2 *d_rows = reinterpret_cast<const int2 *>(matches);
    if (!dev_m) {
        GM_CUDA_R(cudaMemcpyAsync(w, matches, sizeof(int32_t) * 2 * (size_t)M, cudaMemcpyHostToDevice, s));
        d_rows = reinterpret_cast<const int2 *>(w);
        w += m_b;
    } else if (reinterpret_cast<uintptr_t>(matches) % 8 != 0) {
        return fail(GM_ERR_INVALID, "gm_triangulate_image_tracks: device matches must be 8-byte aligned");
    }
    int32_t *flag = reinterpret_cast<int32_t *>(w);
    int32_t *track_of = reinterpret_cast<int32_t *>(w + fl_b);
    int32_t *bsum = reinterpret_cast<int32_t *>(w + fl_b + tr_b);
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(w + fl_b + tr_b + bs_b);
    int64_t *d_pbase = reinterpret_cast<int64_t *>(w + fl_b + tr_b + bs_b + 256);
    int32_t *slot = reinterpret_cast<int32_t *>(w + fl_b + tr_b + bs_b + 256 + pb_b);
    int32_t *cnt = reinterpret_cast<int32_t *>(w + fl_b + tr_b + bs_b + 256 + pb_b + sl_b);
    GM_CUDA_R(cudaMemcpyAsync(d_pbase, pbase.data(), sizeof(int64_t) * (n_pairs + 1), cudaMemcpyHostToDevice, s));
    GM_CUDA_R(cudaMemsetAsync(slot, 0xff, sizeof(int32_t) * (size_t)pbase[n_pairs], s));
    GM_CUDA_R(cudaMemcpyAsync(d_imgs, imgs.data(), sizeof(TriImage) * n_images, cudaMemcpyHostToDevice, s));
    GM_CUDA_R(cudaMemcpyAsync(d_P, P, sizeof(double) * 12 * n_images,
                              dev_p ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    GM_CUDA_R(cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * (n_pairs + 1), cudaMemcpyHostToDevice, s));
    GM_CUDA_R(cudaMemcpyAsync(d_pairs, pairs.data(), sizeof(TrkPair) * n_pairs, cudaMemcpyHostToDevice, s));
    GM_CUDA_R(cudaMemcpyAsync(d_ipoff, img_poff.data(), sizeof(int32_t) * (n_images + 1), cudaMemcpyHostToDevice, s));
    GM_CUDA_R(cudaMemcpyAsync(d_ipairs, img_pairs.data(), sizeof(int32_t) * n_pairs, cudaMemcpyHostToDevice, s));
    GM_CUDA_R(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
    const int grid = std::max(1, ctx->num_sms * 8);
    trk_scatter_kernel<<<grid, 256, 0, s>>>(d_rows, M, d_off, n_pairs, d_pairs, d_imgs, d_pbase, slot, bad);
    trk_count_kernel<<<grid, 256, 0, s>>>(total, d_imgs, n_images, d_ipoff, d_ipairs, d_pbase, slot, flag, cnt);
    GM_CUDA_R(launch_exclusive_scan(flag, (int32_t)total, track_of, bsum, s));
    // one host read for the row check and the track count (the passes above only follow valid rows)
    unsigned long long h_bad = 0;
    int32_t nt = 0;
    GM_CUDA_R(cudaMemcpyAsync(&h_bad, bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s));
    GM_CUDA_R(cudaMemcpyAsync(&nt, track_of + total, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GM_CUDA_R(cudaStreamSynchronize(s));
    if (h_bad)
        return fail(GM_ERR_INVALID,
                    "gm_triangulate_image_tracks: %llu match rows outside their images or not sorted by query", h_bad);
    *n_tracks = nt;
    if (nt > cap) return fail(GM_ERR_NOMEM, "gm_triangulate_image_tracks: %d tracks exceed cap %lld", nt, (long long)cap);
    if (nt == 0) return GM_OK;
    const bool dev_o = is_device_ptr(X);
    if (is_device_ptr(nodes) != dev_o || is_device_ptr(n_views) != dev_o)
        return fail(GM_ERR_INVALID,
                    "gm_triangulate_image_tracks: X, nodes and n_views must all be host or all device memory");
    const size_t x_b = align_up(sizeof(double) * 3 * nt, 256);
    const size_t r_b = align_up(sizeof(int64_t) * nt, 256), v_b = align_up(sizeof(int32_t) * nt, 256);
    if (!dev_o && (st = ensure_dev(ctx, ctx->d_tri_out, x_b + r_b + v_b)) != GM_OK) return st;
    char *o = dev_o ? nullptr : static_cast<char *>(ctx->d_tri_out.p);
    double *dX = dev_o ? X : reinterpret_cast<double *>(o);
    int64_t *dN = dev_o ? nodes : reinterpret_cast<int64_t *>(o + x_b);
    int32_t *dV = dev_o ? n_views : reinterpret_cast<int32_t *>(o + x_b + r_b);
    trk_list_kernel<<<grid, 256, 0, s>>>(total, track_of, dN);
    trk_solve_kernel<<<(unsigned)(((int64_t)nt + kSolveThreads - 1) / kSolveThreads), kSolveThreads, 0, s>>>(
        nt, dN, cnt, d_imgs, n_images, d_ipoff, d_ipairs, d_pairs, d_pbase, slot, d_rows, d_P, dX, dV);
    GM_CUDA_R(cudaGetLastError());
    if (!dev_o) {
        GM_CUDA_R(cudaMemcpyAsync(X, dX, sizeof(double) * 3 * nt, cudaMemcpyDeviceToHost, s));
        GM_CUDA_R(cudaMemcpyAsync(nodes, dN, sizeof(int64_t) * nt, cudaMemcpyDeviceToHost, s));
        GM_CUDA_R(cudaMemcpyAsync(n_views, dV, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost, s));
    }
    GM_CUDA_R(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // extern "C"
