// gm_coarse.cu -- the coarse stage (Sec. 4): high-scale feature selection and the hybrid preemptive two-batch
// matching schedule, run by the batched matcher with an unbounded band.
//
// Views.  For every image the selection is computed on the device: one block per image finds, by an 8-bit radix
// select over 64-bit keys (order-preserving scale bits, then the complemented feature index, so that the key order
// is "larger scale first, then lower index" and every key is distinct), the k-th largest key for k = the first
// batch and k = the kept count; a block-wide compaction then writes the three index lists in ascending feature
// order.  A gather kernel copies the selected features (coordinates, descriptors restored from the resident
// recentred copy, scales) into a staging buffer, from which they are registered as internal images.
// Matching.  The first batch (q1 view of A against the t view of B) runs on the context's workspace; the second
// (q2 view of A) on a second workspace for the pairs whose first batch gave more than min_matches matches; an
// assembly kernel writes both batches' rows in the caller's pair order, mapped back to the images' own indices.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include "gm_ctx.h"

namespace gm {
namespace {

struct Opts {
    int32_t eta, first, min_features, min_matches;
};

struct SelJob {
    const float *scale;             // caller order
    int32_t n, k1, kt;
    int32_t pad_;
    int32_t *q1, *q2, *t;           // outputs: k1, kt - k1 and kt ascending feature indices
};

struct GatherJob {
    const float2 *xy;               // resident image, column-major order
    const int32_t *inv_perm;        // feature index -> column-major position
    const int8_t *desc;             // resident recentred descriptors (bit pattern b ^ 0x80)
    const float *scale;             // caller order
    const int32_t *list;            // view feature -> image feature
    int32_t n, pad_;
    float2 *xy_out;
    uint8_t *desc_out;
    float *scale_out;
};

struct CoarsePairDev {
    int64_t out_off;                // first output row of the pair
    int64_t src1, src2;             // first row of the pair in the first / second batch's rows
    int32_t c1, c2;
    const int32_t *la1, *la2, *lb;  // view feature -> image feature (nullptr = identity)
};

constexpr int kSelThreads = 1024;

__device__ __forceinline__ uint64_t sel_key(float s, int32_t i)
{
    const uint32_t b = s == 0.0f ? 0u : __float_as_uint(s);   // -0 and +0 are the same scale
    const uint32_t o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ((uint64_t)o << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)i);
}

// The k-th largest key of the block's image (1 <= k <= n), most significant digit first.
__device__ uint64_t kth_largest(const float *__restrict__ scale, int32_t n, int32_t k, unsigned int *hist,
                                uint64_t *bcast)
{
    uint64_t prefix = 0, mask = 0;
    int32_t remaining = k;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
        __syncthreads();
        for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint64_t key = sel_key(scale[i], i);
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t cum = 0;
            int d = 255;
            for (; d > 0; --d) {
                if (cum + (int32_t)hist[d] >= remaining) break;
                cum += (int32_t)hist[d];
            }
            remaining -= cum;
            *bcast = prefix | ((uint64_t)d << shift);
        }
        __syncthreads();
        prefix = *bcast;
        mask |= 0xFFull << shift;
    }
    return prefix;
}

__global__ void __launch_bounds__(kSelThreads) select_kernel(const SelJob *__restrict__ jobs,
                                                             unsigned long long *__restrict__ bad)
{
    __shared__ unsigned int hist[256];
    __shared__ uint64_t bcast;
    __shared__ int32_t wsum[3][32];
    __shared__ int32_t base[3], tot[3];
    const SelJob J = jobs[blockIdx.x];
    const uint64_t thr_t = J.kt > 0 ? kth_largest(J.scale, J.n, J.kt, hist, &bcast) : ~0ull;
    const uint64_t thr_1 = J.k1 > 0 ? kth_largest(J.scale, J.n, J.k1, hist, &bcast) : ~0ull;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int lt = (1u << lane) - 1u;
    if (threadIdx.x < 3) base[threadIdx.x] = 0;
    __syncthreads();
    int32_t *out[3] = {J.q1, J.q2, J.t};
    unsigned long long nan_count = 0;
    for (int32_t c0 = 0; c0 < J.n; c0 += kSelThreads) {
        const int32_t i = c0 + threadIdx.x;
        const bool valid = i < J.n;
        const float s = valid ? J.scale[i] : 0.0f;
        if (valid && isnan(s)) ++nan_count;
        const uint64_t key = sel_key(s, i);
        const bool in1 = valid && J.k1 > 0 && key >= thr_1;
        const bool inT = valid && J.kt > 0 && key >= thr_t;
        const bool f[3] = {in1, inT && !in1, inT};
        int32_t pre[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const unsigned int bal = __ballot_sync(0xffffffffu, f[v]);
            pre[v] = __popc(bal & lt);
            if (lane == 0) wsum[v][warp] = __popc(bal);
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const int32_t x = lane < kSelThreads / 32 ? wsum[v][lane] : 0;
                int32_t inc = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                if (lane < kSelThreads / 32) wsum[v][lane] = inc - x;
                if (lane == 31) tot[v] = inc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < 3; ++v)
            if (f[v]) out[v][base[v] + wsum[v][warp] + pre[v]] = i;
        __syncthreads();
        if (threadIdx.x < 3) base[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
    if (nan_count) atomicAdd(&bad[blockIdx.x], nan_count);
}

// One warp per view feature: 128 descriptor bytes as 32 words, coordinates and scale by lane 0.
__global__ void gather_kernel(const GatherJob *__restrict__ jobs)
{
    const GatherJob J = jobs[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int32_t v = blockIdx.x * wpb + (threadIdx.x >> 5); v < J.n; v += gridDim.x * wpb) {
        const int32_t f = J.list[v];
        const int32_t pos = J.inv_perm[f];
        const uint32_t w = reinterpret_cast<const uint32_t *>(J.desc + (size_t)pos * kDim)[lane];
        reinterpret_cast<uint32_t *>(J.desc_out + (size_t)v * kDim)[lane] = w ^ 0x80808080u;
        if (lane == 0) {
            J.xy_out[v] = J.xy[pos];
            J.scale_out[v] = J.scale[f];
        }
    }
}

__global__ void iota_kernel(int32_t *out, int32_t n)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = i;
}

__global__ void assemble_kernel(const CoarsePairDev *__restrict__ P, int32_t n_pairs, int64_t total,
                                const int32_t *__restrict__ rows1, const int32_t *__restrict__ rows2,
                                int32_t *__restrict__ out)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = n_pairs;   // the last pair whose rows start at or before r (pairs without rows share
        while (hi - lo > 1) {           // the next pair's start and come before it)
            const int32_t mid = (lo + hi) >> 1;
            if (P[mid].out_off <= r) lo = mid;
            else hi = mid;
        }
        const CoarsePairDev &p = P[lo];
        int64_t l = r - p.out_off;
        const int32_t *src;
        const int32_t *la;
        if (l < p.c1) {
            src = rows1 + 2 * (p.src1 + l);
            la = p.la1;
        } else {
            l -= p.c1;
            src = rows2 + 2 * (p.src2 + l);
            la = p.la2;
        }
        const int32_t i = src[0], j = src[1];
        out[2 * r] = la ? la[i] : i;
        out[2 * r + 1] = p.lb ? p.lb[j] : j;
    }
}

#define GM_CUDA_C(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return gm::fail(GM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

gm_status resolve_opts(const gm_coarse_opts *opts, Opts &o, const char *fn)
{
    o = Opts{20, 10, 1000, 4};
    if (opts) o = Opts{opts->eta_pct, opts->first_pct, opts->min_features, opts->min_matches};
    if (o.eta < 1 || o.eta > 100 || o.first < 1 || o.first > o.eta || o.min_features < 0 || o.min_matches < 0)
        return fail(GM_ERR_INVALID, "%s: bad options (eta %d, first %d, min_features %d, min_matches %d)", fn, o.eta,
                    o.first, o.min_features, o.min_matches);
    return GM_OK;
}

// Builds the views of every listed image that has none, or stale ones (image put again, other options).
gm_status ensure_views(gm_ctx *ctx, const std::vector<int32_t> &ids, const Opts &o, const char *fn)
{
    std::vector<int32_t> todo;
    for (int32_t id : ids) {
        auto it = ctx->images.find(id);
        if (id < 0 || it == ctx->images.end()) return fail(GM_ERR_NOT_FOUND, "%s: image %d not registered", fn, id);
        const ImageSlot *img = it->second;
        auto cv = ctx->coarse.find(id);
        if (cv != ctx->coarse.end() && cv->second.gen == img->gen && cv->second.eta == o.eta &&
            cv->second.first == o.first && cv->second.min_features == o.min_features)
            continue;
        if (img->dev.n > 0 && !img->has_scale) return fail(GM_ERR_INVALID, "%s: image %d has no scales", fn, id);
        if (std::find(todo.begin(), todo.end(), id) == todo.end()) todo.push_back(id);
    }
    if (todo.empty()) return GM_OK;
    cudaStream_t s = ctx->ws.stream;
    gm_status st;
    std::vector<CoarseViews> nv(todo.size());
    std::vector<SelJob> sel;
    std::vector<size_t> sel_of;   // index into todo of each selection job
    for (size_t u = 0; u < todo.size(); ++u) {
        const ImageSlot *img = ctx->images.at(todo[u]);
        CoarseViews &v = nv[u];
        v.gen = img->gen;
        v.eta = o.eta;
        v.first = o.first;
        v.min_features = o.min_features;
        const int32_t n = img->dev.n;
        if (n < o.min_features) {
            v.all = true;
            v.id[0] = v.id[2] = todo[u];
            v.n[0] = v.n[2] = n;
            continue;
        }
        const int32_t kt = (int32_t)((int64_t)n * o.eta / 100), k1 = (int32_t)((int64_t)n * o.first / 100);
        v.n[0] = k1;
        v.n[1] = kt - k1;
        v.n[2] = kt;
        const size_t b0 = align_up(4 * (size_t)std::max(k1, 1), 256), b1 = align_up(4 * (size_t)std::max(kt - k1, 1), 256);
        if ((st = ensure_dev(ctx, v.lists, b0 + b1 + align_up(4 * (size_t)std::max(kt, 1), 256))) != GM_OK) {
            for (auto &w : nv) free_dev(ctx, w.lists);
            return st;
        }
        char *lp = static_cast<char *>(v.lists.p);
        v.list[0] = reinterpret_cast<int32_t *>(lp);
        v.list[1] = reinterpret_cast<int32_t *>(lp + b0);
        v.list[2] = reinterpret_cast<int32_t *>(lp + b0 + b1);
        SelJob j{};
        j.scale = img->scale;
        j.n = n;
        j.k1 = k1;
        j.kt = kt;
        j.q1 = const_cast<int32_t *>(v.list[0]);
        j.q2 = const_cast<int32_t *>(v.list[1]);
        j.t = const_cast<int32_t *>(v.list[2]);
        sel.push_back(j);
        sel_of.push_back(u);
    }
    auto cleanup = [&]() {
        for (auto &w : nv) free_dev(ctx, w.lists);
    };
    std::vector<gm_image> views;
    std::vector<std::pair<size_t, int>> view_of;   // (todo index, view 0..2) of each registered view
    if (!sel.empty()) {
        const int32_t J = (int32_t)sel.size();
        // selection
        const size_t sel_b = align_up(sizeof(SelJob) * J, 256), bad_b = align_up(sizeof(unsigned long long) * J, 256);
        std::vector<GatherJob> gj;
        size_t stage = 0;
        for (int32_t q = 0; q < J; ++q)
            for (int v = 0; v < 3; ++v) {
                const int32_t n = nv[sel_of[q]].n[v];
                if (n > 0) stage += align_up(8 * (size_t)n, 256) + align_up(128 * (size_t)n, 256) + align_up(4 * (size_t)n, 256);
            }
        const size_t gj_b = align_up(sizeof(GatherJob) * 3 * J, 256);
        if ((st = ensure_dev(ctx, ctx->d_coarse_tab, sel_b + bad_b + gj_b)) != GM_OK) return cleanup(), st;
        if ((st = ensure_dev(ctx, ctx->d_coarse_stage, std::max<size_t>(stage, 256))) != GM_OK) return cleanup(), st;
        char *tab = static_cast<char *>(ctx->d_coarse_tab.p);
        SelJob *d_sel = reinterpret_cast<SelJob *>(tab);
        unsigned long long *d_bad = reinterpret_cast<unsigned long long *>(tab + sel_b);
        GatherJob *d_gj = reinterpret_cast<GatherJob *>(tab + sel_b + bad_b);
        GM_CUDA_C(cudaMemcpyAsync(d_sel, sel.data(), sizeof(SelJob) * J, cudaMemcpyHostToDevice, s));
        GM_CUDA_C(cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long) * J, s));
        select_kernel<<<J, kSelThreads, 0, s>>>(d_sel, d_bad);
        GM_CUDA_C(cudaGetLastError());
        std::vector<unsigned long long> bad(J);
        GM_CUDA_C(cudaMemcpyAsync(bad.data(), d_bad, sizeof(unsigned long long) * J, cudaMemcpyDeviceToHost, s));
        GM_CUDA_C(cudaStreamSynchronize(s));
        for (int32_t q = 0; q < J; ++q)
            if (bad[q]) {
                cleanup();
                return fail(GM_ERR_INVALID, "%s: image %d has %llu NaN scales", fn, todo[sel_of[q]], bad[q]);
            }
        // gather the selected features and register them
        char *sp = static_cast<char *>(ctx->d_coarse_stage.p);
        int32_t max_n = 0;
        for (int32_t q = 0; q < J; ++q) {
            const size_t u = sel_of[q];
            const ImageSlot *img = ctx->images.at(todo[u]);
            for (int v = 0; v < 3; ++v) {
                const int32_t n = nv[u].n[v];
                if (n == 0) continue;
                GatherJob g{};
                g.xy = img->dev.xy;
                g.inv_perm = img->dev.inv_perm;
                g.desc = img->dev.desc;
                g.scale = img->scale;
                g.list = nv[u].list[v];
                g.n = n;
                g.xy_out = reinterpret_cast<float2 *>(sp);
                sp += align_up(8 * (size_t)n, 256);
                g.desc_out = reinterpret_cast<uint8_t *>(sp);
                sp += align_up(128 * (size_t)n, 256);
                g.scale_out = reinterpret_cast<float *>(sp);
                sp += align_up(4 * (size_t)n, 256);
                gj.push_back(g);
                max_n = std::max(max_n, n);
                gm_image im{};
                im.image_id = 0;   // assigned below
                im.width = img->dev.width;
                im.height = img->dev.height;
                im.n = n;
                im.xy = reinterpret_cast<const float *>(g.xy_out);
                im.scale = g.scale_out;
                im.desc = g.desc_out;
                views.push_back(im);
                view_of.push_back({u, v});
            }
        }
        if (!gj.empty()) {
            GM_CUDA_C(cudaMemcpyAsync(d_gj, gj.data(), sizeof(GatherJob) * gj.size(), cudaMemcpyHostToDevice, s));
            for (size_t j0 = 0; j0 < gj.size(); j0 += 65535) {   // grid y: at most 65535 views per launch
                const dim3 grid((unsigned)std::min<int64_t>((max_n + 7) / 8, 1024),
                                (unsigned)std::min<size_t>(gj.size() - j0, 65535));
                gather_kernel<<<grid, 256, 0, s>>>(d_gj + j0);
                GM_CUDA_C(cudaGetLastError());
            }
        }
        // a rebuilt view keeps its internal id, so that its block is reused when large enough
        int32_t fresh_ids = 0;
        for (size_t w = 0; w < views.size(); ++w) {
            auto cv = ctx->coarse.find(todo[view_of[w].first]);
            const int32_t old = cv != ctx->coarse.end() && !cv->second.all ? cv->second.id[view_of[w].second] : 0;
            views[w].image_id = old < 0 ? old : ctx->next_internal_id - fresh_ids++;
        }
        if (!views.empty()) {
            if ((st = put_images(ctx, (int32_t)views.size(), views.data(), 1, fn, true)) != GM_OK) return cleanup(), st;
            ctx->next_internal_id -= fresh_ids;
        }
        for (size_t w = 0; w < views.size(); ++w) nv[view_of[w].first].id[view_of[w].second] = views[w].image_id;
    }
    for (size_t u = 0; u < todo.size(); ++u) {
        auto cv = ctx->coarse.find(todo[u]);
        if (cv != ctx->coarse.end()) {   // the old views not carried over, and the old index lists
            CoarseViews &o = cv->second;
            if (!o.all)
                for (int v = 0; v < 3; ++v)
                    if (o.id[v] < 0 && o.id[v] != nv[u].id[v]) drop_image(ctx, o.id[v]);
            free_dev(ctx, o.lists);
        }
        ctx->coarse[todo[u]] = nv[u];
    }
    return GM_OK;
}

}  // namespace
}  // namespace gm

extern "C" {

gm_status gm_coarse_prepare(gm_ctx *ctx, int32_t n_images, const int32_t *image_ids, const gm_coarse_opts *opts)
{
    using namespace gm;
    if (!ctx || n_images < 0 || (n_images > 0 && !image_ids)) return fail(GM_ERR_INVALID, "gm_coarse_prepare: bad arguments");
    Opts o;
    gm_status st = resolve_opts(opts, o, "gm_coarse_prepare");
    if (st != GM_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA_C(cudaSetDevice(ctx->device));
    return ensure_views(ctx, std::vector<int32_t>(image_ids, image_ids + n_images), o, "gm_coarse_prepare");
}

gm_status gm_coarse_selection(gm_ctx *ctx, int32_t image_id, const gm_coarse_opts *opts, int32_t *q1, int32_t *q2,
                              int32_t *t, int32_t cap, int32_t *counts)
{
    using namespace gm;
    if (!ctx || !counts || cap < 0 || (cap > 0 && (!q1 || !q2 || !t)))
        return fail(GM_ERR_INVALID, "gm_coarse_selection: bad arguments");
    Opts o;
    gm_status st = resolve_opts(opts, o, "gm_coarse_selection");
    if (st != GM_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA_C(cudaSetDevice(ctx->device));
    if ((st = ensure_views(ctx, {image_id}, o, "gm_coarse_selection")) != GM_OK) return st;
    const CoarseViews &v = ctx->coarse.at(image_id);
    for (int k = 0; k < 3; ++k) counts[k] = v.n[k];
    if (std::max({v.n[0], v.n[1], v.n[2]}) > cap)
        return fail(GM_ERR_NOMEM, "gm_coarse_selection: %d indices exceed cap %d", std::max({v.n[0], v.n[1], v.n[2]}),
                    cap);
    cudaStream_t s = ctx->ws.stream;
    int32_t *dst[3] = {q1, q2, t};
    const bool dev = cap > 0 && is_device_ptr(q1);
    if (cap > 0 && (is_device_ptr(q2) != dev || is_device_ptr(t) != dev))
        return fail(GM_ERR_INVALID, "gm_coarse_selection: q1, q2 and t must all be host or all device memory");
    for (int k = 0; k < 3; ++k) {
        if (v.n[k] == 0) continue;
        if (v.all) {
            if (dev) iota_kernel<<<std::max(1, std::min((v.n[k] + 255) / 256, 1024)), 256, 0, s>>>(dst[k], v.n[k]);
            else std::iota(dst[k], dst[k] + v.n[k], 0);
        } else {
            GM_CUDA_C(cudaMemcpyAsync(dst[k], v.list[k], 4 * (size_t)v.n[k], cudaMemcpyDefault, s));
        }
    }
    GM_CUDA_C(cudaGetLastError());
    GM_CUDA_C(cudaStreamSynchronize(s));
    return GM_OK;
}

gm_status gm_match_coarse(gm_ctx *ctx, int32_t n_pairs, const gm_pair *pairs, const gm_coarse_opts *opts,
                          int64_t *pair_off, int32_t *matches, int64_t cap, int64_t *n_written, int32_t *second)
{
    gm::NvtxRange nvtx_("gm_match_coarse");
    using namespace gm;
    const char *fn = "gm_match_coarse";
    if (!ctx || n_pairs < 0 || (n_pairs > 0 && !pairs) || !pair_off || !n_written || cap < 0 || (cap > 0 && !matches))
        return fail(GM_ERR_INVALID, "%s: bad arguments", fn);
    Opts o;
    gm_status st = resolve_opts(opts, o, fn);
    if (st != GM_OK) return st;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA_C(cudaSetDevice(ctx->device));
    *n_written = 0;
    cudaStream_t s = ctx->ws.stream;
    const bool dev_off = is_device_ptr(pair_off);
    if (n_pairs == 0) {
        if (dev_off) GM_CUDA_C(cudaMemset(pair_off, 0, sizeof(int64_t)));
        else pair_off[0] = 0;
        return GM_OK;
    }
    std::vector<int32_t> ids;
    for (int32_t k = 0; k < n_pairs; ++k) {
        if (pairs[k].ratio_den == 0 || pairs[k].ratio_num >= pairs[k].ratio_den)
            return fail(GM_ERR_INVALID, "%s: pair %d: ratio must satisfy 0 <= p < q", fn, k);
        ids.push_back(pairs[k].img_a);
        ids.push_back(pairs[k].img_b);
    }
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    if ((st = ensure_views(ctx, ids, o, fn)) != GM_OK) return st;
    // the first batch
    auto internal_pair = [](const gm_pair &p, int32_t a, int32_t b) {
        gm_pair g = p;
        g.img_a = a;
        g.img_b = b;
        const float F[9] = {0.f, 0.f, 0.f, 0.f, 0.f, -1.f, 0.f, 1.f, 0.f};   // unused: the band is unbounded
        std::memcpy(g.F, F, sizeof(F));
        g.band_px = INFINITY;
        return g;
    };
    std::vector<gm_pair> b1, b2;
    std::vector<int32_t> i1(n_pairs, -1), i2(n_pairs, -1);
    for (int32_t k = 0; k < n_pairs; ++k) {
        const CoarseViews &va = ctx->coarse.at(pairs[k].img_a), &vb = ctx->coarse.at(pairs[k].img_b);
        if (va.n[0] > 0 && vb.n[2] > 0) {
            i1[k] = (int32_t)b1.size();
            b1.push_back(internal_pair(pairs[k], va.id[0], vb.id[2]));
        }
    }
    std::vector<int64_t> off1(b1.size() + 1, 0), off2;
    if (!b1.empty()) {
        if ((st = run_batch(ctx, ctx->ws, (int32_t)b1.size(), b1.data(), true, fn)) != GM_OK) return st;
        std::memcpy(off1.data(), ctx->ws.h_off.p, sizeof(int64_t) * (b1.size() + 1));
    }
    // the second batch: pairs whose first batch gave more than min_matches matches
    for (int32_t k = 0; k < n_pairs; ++k) {
        if (i1[k] < 0) continue;
        const CoarseViews &va = ctx->coarse.at(pairs[k].img_a), &vb = ctx->coarse.at(pairs[k].img_b);
        if (off1[i1[k] + 1] - off1[i1[k]] > o.min_matches && va.n[1] > 0) {
            i2[k] = (int32_t)b2.size();
            b2.push_back(internal_pair(pairs[k], va.id[1], vb.id[2]));
        }
    }
    off2.assign(b2.size() + 1, 0);
    if (!b2.empty()) {
        if ((st = run_batch(ctx, ctx->ws2, (int32_t)b2.size(), b2.data(), true, fn)) != GM_OK) return st;
        std::memcpy(off2.data(), ctx->ws2.h_off.p, sizeof(int64_t) * (b2.size() + 1));
    }
    // offsets, flags and the assembly table
    std::vector<int64_t> off(n_pairs + 1, 0);
    std::vector<CoarsePairDev> tab(n_pairs);
    std::vector<int32_t> flag(n_pairs, 0);
    for (int32_t k = 0; k < n_pairs; ++k) {
        const CoarseViews &va = ctx->coarse.at(pairs[k].img_a), &vb = ctx->coarse.at(pairs[k].img_b);
        CoarsePairDev &p = tab[k];
        p.out_off = off[k];
        p.src1 = i1[k] >= 0 ? off1[i1[k]] : 0;
        p.c1 = i1[k] >= 0 ? (int32_t)(off1[i1[k] + 1] - off1[i1[k]]) : 0;
        p.src2 = i2[k] >= 0 ? off2[i2[k]] : 0;
        p.c2 = i2[k] >= 0 ? (int32_t)(off2[i2[k] + 1] - off2[i2[k]]) : 0;
        p.la1 = va.all ? nullptr : va.list[0];
        p.la2 = va.all ? nullptr : va.list[1];
        p.lb = vb.all ? nullptr : vb.list[2];
        flag[k] = i2[k] >= 0;
        off[k + 1] = off[k] + p.c1 + p.c2;
    }
    const int64_t total = off[n_pairs];
    *n_written = total;
    if (dev_off) GM_CUDA_C(cudaMemcpyAsync(pair_off, off.data(), sizeof(int64_t) * (n_pairs + 1), cudaMemcpyHostToDevice, s));
    else std::memcpy(pair_off, off.data(), sizeof(int64_t) * (n_pairs + 1));
    if (second) {
        if (is_device_ptr(second))
            GM_CUDA_C(cudaMemcpyAsync(second, flag.data(), sizeof(int32_t) * n_pairs, cudaMemcpyHostToDevice, s));
        else
            std::memcpy(second, flag.data(), sizeof(int32_t) * n_pairs);
    }
    if (total > cap) {
        GM_CUDA_C(cudaStreamSynchronize(s));
        return fail(GM_ERR_NOMEM, "%s: %lld matches exceed cap %lld", fn, (long long)total, (long long)cap);
    }
    if (total > 0) {
        const bool dev_m = is_device_ptr(matches);
        const size_t tab_b = align_up(sizeof(CoarsePairDev) * n_pairs, 256);
        if ((st = ensure_dev(ctx, ctx->d_coarse_tab, tab_b)) != GM_OK) return st;
        if (!dev_m && (st = ensure_dev(ctx, ctx->d_coarse_out, sizeof(int32_t) * 2 * (size_t)total)) != GM_OK) return st;
        CoarsePairDev *d_tab = static_cast<CoarsePairDev *>(ctx->d_coarse_tab.p);
        int32_t *dst = dev_m ? matches : static_cast<int32_t *>(ctx->d_coarse_out.p);
        GM_CUDA_C(cudaMemcpyAsync(d_tab, tab.data(), sizeof(CoarsePairDev) * n_pairs, cudaMemcpyHostToDevice, s));
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 8));
        assemble_kernel<<<grid, 256, 0, s>>>(d_tab, n_pairs, total, static_cast<const int32_t *>(ctx->ws.d_rows.p),
                                             static_cast<const int32_t *>(ctx->ws2.d_rows.p), dst);
        GM_CUDA_C(cudaGetLastError());
        if (!dev_m) GM_CUDA_C(cudaMemcpyAsync(matches, dst, sizeof(int32_t) * 2 * total, cudaMemcpyDeviceToHost, s));
    }
    GM_CUDA_C(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // extern "C"
