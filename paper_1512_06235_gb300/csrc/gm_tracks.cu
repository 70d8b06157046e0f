// gm_tracks.cu -- gm_merge_tracks: tracks as the connected components of the feature matches (the track merging
// step after pairwise matching, Sec. 6.2).
//
// Nodes are features (one global index per (image, feature)), matches are undirected edges.  A lock-free
// union-find runs on the device: every edge links the roots of its endpoints, always the larger root under the
// smaller (compare-and-swap on the larger root's parent), so the root of every tree is its smallest node; finds
// halve their paths.  Afterwards every node's label is its root, i.e. the smallest node index of its component,
// whatever order the links happened in.  Parent reads bypass L1 (volatile) so that a retrying link sees other
// SMs' links; every retry loop is bounded and reports an error when the bound is hit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "gm_ctx.h"

namespace gm {

bool is_device_ptr(const void *p);

namespace {

constexpr int kMaxSteps = 1 << 22;   // bound on the steps of one find or one link retry loop

__device__ __forceinline__ int64_t ld_parent(const int64_t *parent, int64_t x)
{
    return *reinterpret_cast<const volatile int64_t *>(parent + x);
}

// root of x with path halving; -1 if the step bound is hit
__device__ __forceinline__ int64_t find_root(int64_t *parent, int64_t x)
{
    for (int it = 0; it < kMaxSteps; ++it) {
        const int64_t p = ld_parent(parent, x);
        if (p == x) return x;
        const int64_t gp = ld_parent(parent, p);
        if (gp != p) *reinterpret_cast<volatile int64_t *>(parent + x) = gp;   // still an ancestor of x
        x = gp;
    }
    return -1;
}

__global__ void init_kernel(int64_t *parent, int64_t n)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = v;
}

__global__ void link_kernel(const int64_t *__restrict__ edges, int64_t n_edges, int64_t n_nodes, int64_t *parent,
                            unsigned long long *bad)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= n_nodes || v >= n_nodes) {
            atomicAdd(&bad[0], 1ull);
            continue;
        }
        bool done = false;
        for (int it = 0; it < kMaxSteps && !done; ++it) {
            u = find_root(parent, u);
            v = find_root(parent, v);
            if (u < 0 || v < 0) break;
            if (u == v) {
                done = true;
                break;
            }
            const int64_t hi = max(u, v), lo = min(u, v);
            const unsigned long long prev =
                atomicCAS(reinterpret_cast<unsigned long long *>(parent + hi), (unsigned long long)hi,
                          (unsigned long long)lo);
            done = prev == (unsigned long long)hi;   // hi was still a root: linked; otherwise retry from the new roots
        }
        if (!done) atomicAdd(&bad[1], 1ull);
    }
}

// labels: the root of every node; a non-root member marks its root, whose track is counted once
__global__ void label_kernel(int64_t *parent, int64_t n, int64_t *labels, unsigned int *member_of,
                             unsigned long long *bad)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = find_root(parent, v);
        if (r < 0) {
            atomicAdd(&bad[1], 1ull);
            labels[v] = v;
            continue;
        }
        labels[v] = r;
        if (r != v) member_of[r] = 1u;
    }
}

__global__ void count_kernel(const unsigned int *__restrict__ member_of, int64_t n, unsigned long long *n_tracks)
{
    unsigned long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        c += member_of[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n_tracks, c);
}

#define GM_CUDA_K(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return gm::fail(GM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace
}  // namespace gm

extern "C" {

gm_status gm_merge_tracks(gm_ctx *ctx, int64_t n_nodes, int64_t n_edges, const int64_t *edges, int64_t *labels,
                          int64_t *n_tracks)
{
    gm::NvtxRange nvtx_("gm_merge_tracks");
    using namespace gm;
    if (!ctx || n_nodes < 0 || n_edges < 0 || (n_edges > 0 && !edges) || (n_nodes > 0 && !labels) || !n_tracks)
        return fail(GM_ERR_INVALID, "gm_merge_tracks: bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA_K(cudaSetDevice(ctx->device));
    *n_tracks = 0;
    if (n_nodes == 0) {
        if (n_edges > 0) return fail(GM_ERR_INVALID, "gm_merge_tracks: edges without nodes");
        return GM_OK;
    }
    cudaStream_t s = ctx->ws.stream;
    const bool dev_e = n_edges == 0 || is_device_ptr(edges), dev_l = is_device_ptr(labels);
    const size_t par_b = align_up(sizeof(int64_t) * (size_t)n_nodes, 256);
    const size_t lab_b = dev_l ? 0 : par_b;
    const size_t mem_b = align_up(sizeof(unsigned int) * (size_t)n_nodes, 256);
    const size_t edg_b = dev_e ? 0 : align_up(sizeof(int64_t) * 2 * (size_t)n_edges, 256);
    gm_status st = ensure_dev(ctx, ctx->d_tracks, par_b + lab_b + mem_b + edg_b + 256);
    if (st != GM_OK) return st;
    char *w = static_cast<char *>(ctx->d_tracks.p);
    int64_t *parent = reinterpret_cast<int64_t *>(w);
    int64_t *lab = dev_l ? labels : reinterpret_cast<int64_t *>(w + par_b);
    unsigned int *member_of = reinterpret_cast<unsigned int *>(w + par_b + lab_b);
    const int64_t *d_edges = edges;
    if (!dev_e) {
        int64_t *de = reinterpret_cast<int64_t *>(w + par_b + lab_b + mem_b);
        GM_CUDA_K(cudaMemcpyAsync(de, edges, sizeof(int64_t) * 2 * (size_t)n_edges, cudaMemcpyHostToDevice, s));
        d_edges = de;
    }
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(w + par_b + lab_b + mem_b + edg_b);
    GM_CUDA_K(cudaMemsetAsync(ctr, 0, 3 * sizeof(unsigned long long), s));
    GM_CUDA_K(cudaMemsetAsync(member_of, 0, sizeof(unsigned int) * (size_t)n_nodes, s));
    const int grid = std::max(1, ctx->num_sms * 8);
    init_kernel<<<grid, 256, 0, s>>>(parent, n_nodes);
    if (n_edges > 0) link_kernel<<<grid, 256, 0, s>>>(d_edges, n_edges, n_nodes, parent, ctr);
    label_kernel<<<grid, 256, 0, s>>>(parent, n_nodes, lab, member_of, ctr);
    count_kernel<<<grid, 256, 0, s>>>(member_of, n_nodes, ctr + 2);
    GM_CUDA_K(cudaGetLastError());
    unsigned long long h[3] = {0, 0, 0};
    GM_CUDA_K(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
    if (!dev_l)
        GM_CUDA_K(cudaMemcpyAsync(labels, lab, sizeof(int64_t) * (size_t)n_nodes, cudaMemcpyDeviceToHost, s));
    GM_CUDA_K(cudaStreamSynchronize(s));
    if (h[0]) return fail(GM_ERR_INVALID, "gm_merge_tracks: %llu edges have an endpoint outside [0, %lld)", h[0],
                          (long long)n_nodes);
    if (h[1]) return fail(GM_ERR_TIMEOUT, "gm_merge_tracks: %llu link or find loops hit their bound", h[1]);
    *n_tracks = (int64_t)h[2];
    return GM_OK;
}

}  // extern "C"
