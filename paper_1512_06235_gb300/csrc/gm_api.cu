// gm_api.cu -- host side of libgeomatch: the C ABI declared in include/geomatch.h.
//
// A context owns one CUDA stream, the resident images (binned once, App. A Step 1) and a grow-only workspace.
// gm_match_pairs runs a whole batch of pairs with a fixed number of launches, independent of the number of
// pairs (Sec. 6.2.3: pairs are independent; App. A Steps 2-4 for all pairs at once):
//   H2D pair table -> order kernel (one block per pair) -> match kernel (all pairs' queries) -> count + scan ->
//   write -> D2H of the offsets -> copy of the match rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "gm_ctx.h"

using namespace gm;

namespace gm {
namespace {
thread_local std::string g_err = "";
// After the 64 counter shards of a batch: the persistent kernels' work-queue counter (int32 in the first 8 bytes),
// the candidate-stream entries used, and the tcgen05 grid's three timing words (launch_match_tc).
constexpr size_t kCtrTail = 5 * sizeof(unsigned long long);
}  // namespace

gm_status fail(gm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

const char *last_error() { return g_err.c_str(); }

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

#define GM_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return gm::fail(GM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

gm_status ensure_dev(gm_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (b.bytes >= bytes) return GM_OK;
    size_t nb = align_up(std::max({bytes, b.bytes + b.bytes / 2, (size_t)256}), 256);
    const size_t others = ctx->bytes_images + ctx->bytes_work - b.bytes;
    if (ctx->budget && others + nb > ctx->budget) {
        nb = align_up(bytes, 256);
        if (others + nb > ctx->budget)
            return fail(GM_ERR_BUDGET, "workspace of %zu bytes exceeds the device-memory budget", nb);
    }
    free_dev(ctx, b);
    if (cudaMalloc(&b.p, nb) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(GM_ERR_NOMEM, "cudaMalloc of %zu bytes failed", nb);
    }
    b.bytes = nb;
    ctx->bytes_work += nb;
    return GM_OK;
}

gm_status ensure_host(HostBuf &b, size_t bytes, bool mapped)
{
    if (b.bytes >= bytes && b.mapped == mapped) return GM_OK;
    const size_t nb = align_up(std::max(bytes, b.bytes + b.bytes / 2), 4096);
    free_host(b);
    if (cudaHostAlloc(&b.p, nb, mapped ? cudaHostAllocMapped : cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(GM_ERR_NOMEM, "cudaHostAlloc of %zu bytes failed", nb);
    }
    b.bytes = nb;
    b.mapped = mapped;
    return GM_OK;
}

void free_dev(gm_ctx *ctx, DevBuf &b)
{
    if (b.p) {
        cudaFree(b.p);
        ctx->bytes_work -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

void free_host(HostBuf &b)
{
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

gm_status workspace_init(Workspace &ws, cudaStream_t stream)
{
    if (stream) {
        ws.stream = stream;
        ws.own_stream = false;
    } else {
        GM_CUDA(cudaStreamCreateWithFlags(&ws.stream, cudaStreamNonBlocking));
        ws.own_stream = true;
    }
    for (auto &e : ws.ev) GM_CUDA(cudaEventCreate(&e));
    return GM_OK;
}

void workspace_free(gm_ctx *ctx, Workspace &ws)
{
    if (ws.stream) cudaStreamSynchronize(ws.stream);
    for (DevBuf *b : {&ws.d_tab, &ws.d_qorder, &ws.d_matchj, &ws.d_counts, &ws.d_off, &ws.d_rows, &ws.d_ctr, &ws.d_next,
                      &ws.d_grec, &ws.d_grows, &ws.d_stream})
        free_dev(ctx, *b);
    for (HostBuf *b : {&ws.h_tab, &ws.h_off, &ws.h_rows}) free_host(*b);
    if (ws.gexec) cudaGraphExecDestroy(ws.gexec);
    ws.gexec = nullptr;
    for (auto &e : ws.ev)
        if (e) cudaEventDestroy(e);
    if (ws.own_stream && ws.stream) cudaStreamDestroy(ws.stream);
    ws.stream = nullptr;
}

size_t workspace_bytes(const Workspace &ws)
{
    size_t n = 0;
    for (const DevBuf *b : {&ws.d_tab, &ws.d_qorder, &ws.d_matchj, &ws.d_counts, &ws.d_off, &ws.d_rows, &ws.d_ctr,
                            &ws.d_next, &ws.d_grec, &ws.d_grows, &ws.d_stream})
        n += b->bytes;
    return n;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device memory of the given device, or managed memory (which every device may access).
bool is_device_ptr_on(const void *p, int device)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == device);
}

// The device address of page-locked host memory that the device may read directly (cudaMallocHost /
// cudaHostAlloc / mapped registrations), or nullptr for any other pointer (pageable memory is always copied).
const void *mapped_host_ptr(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

namespace {

struct CopySeg {
    const void *src;
    void *dst;
    int64_t words;              // 4-byte words
};

// Copies of 4-byte-aligned segments (blockIdx.y: segment), e.g. from mapped host memory into image blocks.
__global__ void copy_segments_kernel(const CopySeg *__restrict__ segs)
{
    const CopySeg g = segs[blockIdx.y];
    const uint32_t *src = static_cast<const uint32_t *>(g.src);
    uint32_t *dst = static_cast<uint32_t *>(g.dst);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.words; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

}  // namespace

gm_status prepare_pair(gm_ctx *ctx, const gm_pair &pr, int64_t k, PairDev &pd, bool internal)
{
    if (!internal && (pr.img_a < 0 || pr.img_b < 0))
        return fail(GM_ERR_NOT_FOUND, "pair %lld: image %d not registered", (long long)k, std::min(pr.img_a, pr.img_b));
    auto ia = ctx->images.find(pr.img_a), ib = ctx->images.find(pr.img_b);
    if (ia == ctx->images.end() || ib == ctx->images.end())
        return fail(GM_ERR_NOT_FOUND, "pair %lld: image %d not registered", (long long)k,
                    ia == ctx->images.end() ? pr.img_a : pr.img_b);
    for (int t = 0; t < 9; ++t)
        if (!std::isfinite(pr.F[t])) return fail(GM_ERR_INVALID, "pair %lld: F is not finite", (long long)k);
    if (std::isnan(pr.band_px) || pr.band_px < 0.0f)
        return fail(GM_ERR_INVALID, "pair %lld: band_px must be >= 0 or +inf", (long long)k);
    if (pr.ratio_den == 0 || pr.ratio_num >= pr.ratio_den)
        return fail(GM_ERR_INVALID, "pair %lld: ratio must satisfy 0 <= p < q", (long long)k);
    pd.a = ia->second->slot;
    pd.b = ib->second->slot;
    std::memcpy(pd.F, pr.F, sizeof(pd.F));
    pd.d = pr.band_px;
    pd.p = pr.ratio_num;
    pd.q = pr.ratio_den;
    pd.n_a = ia->second->dev.n;
    pd.flags = 0;
    pd.qoff = 0;
    return GM_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time dependency on libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Descriptor rows: fp16 [n][128], box 64 x 64 (128-byte swizzle).  Records: [n + 1][4] read as FP32, box 4 x 64,
// out-of-range rows filled with NaN.
gm_status encode_maps(const ImageDev &dev, TmaMaps &maps)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(GM_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const cuuint32_t estride[2] = {1, 1};
    const cuuint64_t dims[2] = {(cuuint64_t)kDim, (cuuint64_t)dev.n};
    const cuuint64_t strides[1] = {(cuuint64_t)kDim * 2};
    const cuuint32_t box[2] = {64, 64};
    if (enc(&maps.desc_tile, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<uint16_t *>(dev.desc_h), dims, strides, box,
            estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(GM_ERR_CUDA, "cuTensorMapEncodeTiled failed (descriptor tiles)");
    const cuuint32_t rowbox[2] = {64, 1};
    if (enc(&maps.desc_row, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<uint16_t *>(dev.desc_h), dims, strides,
            rowbox, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(GM_ERR_CUDA, "cuTensorMapEncodeTiled failed (descriptor rows)");
    const cuuint64_t rdims[2] = {4, (cuuint64_t)dev.n + 1};
    const cuuint64_t rstrides[1] = {16};
    const cuuint32_t rbox[2] = {4, 64};
    if (enc(&maps.rec_tile, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<int4 *>(dev.rec), rdims, rstrides, rbox,
            estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA) != CUDA_SUCCESS)
        return fail(GM_ERR_CUDA, "cuTensorMapEncodeTiled failed (records)");
    const cuuint64_t xdims[2] = {16, (cuuint64_t)dev.n};
    const cuuint64_t xstrides[1] = {32};
    const cuuint32_t xbox[2] = {16, 64};
    if (enc(&maps.ext_tile, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<uint16_t *>(dev.ext_h), xdims, xstrides, xbox,
            estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(GM_ERR_CUDA, "cuTensorMapEncodeTiled failed (norm rows)");
    return GM_OK;
}

gm_status engine_plan(gm_ctx *ctx, Workspace &ws, int32_t n_pairs, const gm_pair *pairs, bool internal)
{
    ws.pd.resize(n_pairs);
    ws.n_pairs = n_pairs;
    ws.Q = 0;
    ws.nitems = 0;
    ws.max_lines = 1;
    ws.whole_image = n_pairs > 0;
    for (int32_t k = 0; k < n_pairs; ++k) {
        gm_status st = prepare_pair(ctx, pairs[k], k, ws.pd[k], internal);
        if (st != GM_OK) return st;
        ImageSlot *sa = ctx->slots[ws.pd[k].a], *sb = ctx->slots[ws.pd[k].b];
        sa->last_use = sb->last_use = ++ctx->use_tick;
        ws.max_lines = std::max(ws.max_lines, std::max(sb->dev.gx, sb->dev.gy));
        ws.whole_image = ws.whole_image && std::isinf(ws.pd[k].d);
        ws.pd[k].qoff = ws.Q;
        ws.Q += ws.pd[k].n_a;
        ws.nitems += (ws.pd[k].n_a + kQueriesPerItem - 1) / kQueriesPerItem;
    }
    if (ws.nitems > INT32_MAX / 2 || ws.Q > INT32_MAX / 2) return fail(GM_ERR_INVALID, "batch too large");
    return GM_OK;
}

gm_status engine_launch(gm_ctx *ctx, Workspace &ws, int32_t *rows_dst)
{
    const int32_t P = ws.n_pairs;
    const int64_t Q = ws.Q;
    const size_t pair_bytes = align_up(sizeof(PairDev) * std::max(P, 1), 256);
    const size_t tab_bytes = 2 * pair_bytes + sizeof(int64_t) * (P + 1);
    gm_status st;
    if ((st = ensure_dev(ctx, ws.d_tab, tab_bytes)) != GM_OK) return st;
    if ((st = ensure_dev(ctx, ws.d_qorder, sizeof(int32_t) * std::max<int64_t>(Q, 1))) != GM_OK) return st;
    if ((st = ensure_dev(ctx, ws.d_matchj, sizeof(int32_t) * std::max<int64_t>(Q, 1))) != GM_OK) return st;
    if ((st = ensure_dev(ctx, ws.d_counts, sizeof(int32_t) * std::max(P, 1))) != GM_OK) return st;
    if ((st = ensure_dev(ctx, ws.d_off, sizeof(int64_t) * (P + 1))) != GM_OK) return st;
    if (!rows_dst && (st = ensure_dev(ctx, ws.d_rows, sizeof(int32_t) * 2 * std::max<int64_t>(Q, 1))) != GM_OK)
        return st;
    if ((st = ensure_dev(ctx, ws.d_ctr, sizeof(BatchCounters) * 64 + 256)) != GM_OK) return st;
    if ((st = ensure_host(ws.h_tab, tab_bytes)) != GM_OK) return st;
    if ((st = ensure_host(ws.h_off, sizeof(int64_t) * (P + 1) + sizeof(BatchCounters) * 64 + kCtrTail)) != GM_OK)
        return st;

    // distance path and work-item size
    int path = ctx->path == GM_PATH_AUTO ? GM_PATH_TC : ctx->path;
    const int32_t max_lines = ws.max_lines;   // longest grid line count of the batch's target images (planned)
    // the tcgen05 kernel's run table holds match_tc_max_grid_lines() grid lines
    if (path == GM_PATH_TC && max_lines > match_tc_max_grid_lines()) path = GM_PATH_MMA;
    // every pair with d = inf: the whole-image specialisation of the tcgen05 kernel
    const bool whole_image = ws.whole_image;
    const int mt = ctx->mma_mt;
    const int qpi = path == GM_PATH_SIMT ? kQueriesPerItem : path == GM_PATH_TC ? kTcQueriesPerItem : 16 * mt;

    char *hs = static_cast<char *>(ws.h_tab.p);
    std::memcpy(hs, ws.pd.data(), sizeof(PairDev) * P);
    // processing order: pairs grouped by image B (then A), so that the groups in flight at the same time read the
    // same B descriptors and these stay in L2; results stay indexed by the caller's pair order
    // (two stable counting sorts over the image slots, by A then by B: linear in the pairs, where a comparison sort
    // of the 72-byte records cost over a millisecond of host time per 20000 pairs with the device idle)
    {
        int32_t n_slots = 1;
        for (const PairDev &pd : ws.pd) n_slots = std::max(n_slots, std::max(pd.a, pd.b) + 1);
        ws.proc.resize(P);
        ws.sort_tmp.resize(P);
        ws.sort_cnt.assign((size_t)n_slots + 1, 0);
        for (int32_t k = 0; k < P; ++k) ++ws.sort_cnt[ws.pd[k].a + 1];
        for (int32_t t = 0; t < n_slots; ++t) ws.sort_cnt[t + 1] += ws.sort_cnt[t];
        for (int32_t k = 0; k < P; ++k) ws.sort_tmp[ws.sort_cnt[ws.pd[k].a]++] = k;
        ws.sort_cnt.assign((size_t)n_slots + 1, 0);
        for (int32_t k = 0; k < P; ++k) ++ws.sort_cnt[ws.pd[k].b + 1];
        for (int32_t t = 0; t < n_slots; ++t) ws.sort_cnt[t + 1] += ws.sort_cnt[t];
        for (int32_t k = 0; k < P; ++k) {
            const int32_t x = ws.sort_tmp[k];
            ws.proc[ws.sort_cnt[ws.pd[x].b]++] = x;
        }
    }
    PairDev *h_proc = reinterpret_cast<PairDev *>(hs + pair_bytes);
    for (int32_t k = 0; k < P; ++k) h_proc[k] = ws.pd[ws.proc[k]];
    int64_t *h_item_off = reinterpret_cast<int64_t *>(hs + 2 * pair_bytes);
    h_item_off[0] = 0;
    for (int32_t k = 0; k < P; ++k) h_item_off[k + 1] = h_item_off[k] + (h_proc[k].n_a + qpi - 1) / qpi;

    char *ds = static_cast<char *>(ws.d_tab.p);
    const PairDev *d_pairs = reinterpret_cast<const PairDev *>(ds);                  // caller's order
    const PairDev *d_proc = reinterpret_cast<const PairDev *>(ds + pair_bytes);      // processing order
    const int64_t *d_item_off = reinterpret_cast<const int64_t *>(ds + 2 * pair_bytes);
    int32_t *qorder = static_cast<int32_t *>(ws.d_qorder.p);
    int32_t *match_j = static_cast<int32_t *>(ws.d_matchj.p);
    BatchCounters *ctr = static_cast<BatchCounters *>(ws.d_ctr.p);
    int32_t *next = reinterpret_cast<int32_t *>(ctr + 64);
    unsigned long long *stream_used = reinterpret_cast<unsigned long long *>(ctr + 64) + 1;
    unsigned long long *cta_time = reinterpret_cast<unsigned long long *>(ctr + 64) + 2;
    const ImageDev *imgs = static_cast<const ImageDev *>(ctx->d_imgs.p);
    int64_t *d_off = static_cast<int64_t *>(ws.d_off.p);
    int32_t *rows = rows_dst ? rows_dst : static_cast<int32_t *>(ws.d_rows.p);
    cudaStream_t s = ws.stream;
    const int64_t n_items = h_item_off[P];
    if (path == GM_PATH_TC) {
        if ((st = ensure_dev(ctx, ws.d_grec, sizeof(GroupDesc) * std::max<int64_t>(n_items, 1))) != GM_OK) return st;
        if ((st = ensure_dev(ctx, ws.d_grows, sizeof(int32_t) * kTcQueriesPerItem * std::max<int64_t>(n_items, 1))) !=
            GM_OK)
            return st;
        if (ws.stream_cap == 0) ws.stream_cap = std::max<int64_t>(1 << 22, 8 * Q);
        if ((st = ensure_dev(ctx, ws.d_stream, sizeof(int32_t) * ws.stream_cap)) != GM_OK) return st;
        ws.stream_cap = (int64_t)(ws.d_stream.bytes / sizeof(int32_t));
    }
    if (ctx->num_sms <= 0) ctx->num_sms = 1;
    const int bps = path == GM_PATH_SIMT ? match_simt_blocks_per_sm()
                    : path == GM_PATH_TC ? match_tc_blocks_per_sm() : match_mma_blocks_per_sm(mt);
    const int32_t grid = ctx->num_sms * bps;
    auto launch_match = [&](int64_t i0, int64_t i1, int32_t gsz) -> cudaError_t {
        if (path == GM_PATH_SIMT)
            return launch_match_simt(imgs, d_proc, d_item_off, P, qorder, i0, i1, gsz, next, match_j, ctr, s);
        if (path == GM_PATH_TC)
            return launch_match_tc(static_cast<const TmaMaps *>(ctx->d_maps.p),
                                   static_cast<const GroupDesc *>(ws.d_grec.p),
                                   static_cast<const int32_t *>(ws.d_grows.p), static_cast<const int32_t *>(ws.d_stream.p),
                                   i0, i1, gsz > 0 ? gsz : ctx->num_sms, match_j, ctr, cta_time, whole_image,
                                   ctx->tc_pipe, s);
        return launch_match_mma(mt, imgs, d_proc, d_item_off, P, qorder, i0, i1, gsz, next, match_j, ctr, s);
    };

    // everything below is stream work only; with GM_OPT_GRAPH it is captured once per batch shape (sizes, launch
    // geometry and every buffer address) and replayed when the shape repeats: the pinned tables it copies from are
    // rewritten above before every replay
    auto enqueue = [&](bool capturing) -> gm_status {
        auto record = [&](cudaEvent_t e) {
            return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
        };
        ws.launches = 0;
        GM_CUDA(record(ws.ev[0]));
        GM_CUDA(cudaMemcpyAsync(ds, hs, tab_bytes, cudaMemcpyHostToDevice, s));
        GM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(BatchCounters) * 64 + kCtrTail, s));
        if (ctx->schedule == 1) {
            // plain form: every pair gets its own launches (one block per work item)
            GM_CUDA(record(ws.ev[1]));
            for (int32_t k = 0; k < P; ++k) {
                GM_CUDA(launch_order(imgs, d_proc + k, 1, qorder, s));
                if (path == GM_PATH_TC) {
                    GM_CUDA(launch_stream(imgs, d_proc, d_item_off, P, qorder, h_item_off[k], h_item_off[k + 1],
                                          static_cast<GroupDesc *>(ws.d_grec.p), static_cast<int32_t *>(ws.d_grows.p),
                                          static_cast<int32_t *>(ws.d_stream.p), ws.stream_cap, stream_used, ctr,
                                          max_lines, s));
                    ++ws.launches;
                }
                GM_CUDA(launch_match(h_item_off[k], h_item_off[k + 1], 0));
                ws.launches += 1 + (h_item_off[k + 1] > h_item_off[k]);
            }
            GM_CUDA(record(ws.ev[2]));
        } else {
            GM_CUDA(launch_order(imgs, d_proc, P, qorder, s));
            if (path == GM_PATH_TC) {
                GM_CUDA(launch_stream(imgs, d_proc, d_item_off, P, qorder, 0, n_items,
                                      static_cast<GroupDesc *>(ws.d_grec.p), static_cast<int32_t *>(ws.d_grows.p),
                                      static_cast<int32_t *>(ws.d_stream.p), ws.stream_cap, stream_used, ctr,
                                      max_lines, s));
                ++ws.launches;
            }
            GM_CUDA(record(ws.ev[1]));
            GM_CUDA(launch_match(0, h_item_off[P], grid));
            GM_CUDA(record(ws.ev[2]));
            ws.launches += 2;
        }
        GM_CUDA(launch_count_matches(d_pairs, P, match_j, static_cast<int32_t *>(ws.d_counts.p), d_off, s));
        GM_CUDA(launch_write_matches(d_pairs, P, match_j, d_off, rows, s));
        ws.launches += 3;
        GM_CUDA(record(ws.ev[3]));
        int64_t *h_off = static_cast<int64_t *>(ws.h_off.p);
        BatchCounters *h_ctr = reinterpret_cast<BatchCounters *>(h_off + P + 1);
        GM_CUDA(cudaMemcpyAsync(h_off, d_off, sizeof(int64_t) * (P + 1), cudaMemcpyDeviceToHost, s));
        GM_CUDA(cudaMemcpyAsync(h_ctr, ctr, sizeof(BatchCounters) * 64 + kCtrTail, cudaMemcpyDeviceToHost, s));
        return GM_OK;
    };
    ws.path_used = path;
    if (!ctx->graph || ctx->schedule == 1) return enqueue(false);
    const GraphKey key{P, Q, n_items, path, mt, ctx->tc_pipe, 0, grid, ws.stream_cap, tab_bytes, ws.d_tab.p, ws.d_qorder.p,
                       ws.d_matchj.p, ws.d_counts.p, ws.d_off.p, rows, ws.d_ctr.p, ws.d_grec.p, ws.d_grows.p,
                       ws.d_stream.p, ctx->d_imgs.p, ctx->d_maps.p, ws.h_tab.p, ws.h_off.p, s};
    if (ws.gexec && std::memcmp(&key, &ws.gkey, sizeof(key)) == 0) {
        GM_CUDA(cudaGraphLaunch(ws.gexec, s));
        ws.launches = ws.glaunches;
        return GM_OK;
    }
    if (std::memcmp(&key, &ws.gseen, sizeof(key)) != 0) {   // a new shape runs directly once; captured when seen again
        ws.gseen = key;
        return enqueue(false);
    }
    if (ws.gexec) {
        cudaGraphExecDestroy(ws.gexec);
        ws.gexec = nullptr;
    }
    GM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const gm_status est = enqueue(true);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (est != GM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return est;
    }
    if (ce != cudaSuccess) return fail(GM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&ws.gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        ws.gexec = nullptr;
        return fail(GM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
    }
    ws.gkey = key;
    ws.glaunches = ws.launches;
    GM_CUDA(cudaGraphLaunch(ws.gexec, s));
    return GM_OK;
}

void engine_stats(gm_ctx *ctx, Workspace &ws, gm_stats &S)
{
    const int32_t P = ws.n_pairs;
    const int64_t *h_off = static_cast<const int64_t *>(ws.h_off.p);
    const BatchCounters *h_ctr = reinterpret_cast<const BatchCounters *>(h_off + P + 1);
    S = gm_stats{};
    S.n_pairs = P;
    S.n_queries = ws.Q;
    for (int k = 0; k < 64; ++k) {
        S.n_candidates += (int64_t)h_ctr[k].candidates;
        S.n_examined += (int64_t)h_ctr[k].examined;
        S.n_redecided += (int64_t)h_ctr[k].redecided;
    }
    S.n_matches = h_off[P];
    for (int k = 0; k < 64; ++k) {
        S.n_device_errors += (int64_t)h_ctr[k].errors;
        S.n_unstaged_groups += (int64_t)h_ctr[k].unstaged;
    }
    ws.overflow = 0;
    for (int k = 0; k < 64; ++k) ws.overflow += (int64_t)h_ctr[k].overflow;
    const unsigned long long *tail = reinterpret_cast<const unsigned long long *>(h_ctr + 64);
    ws.stream_used = (int64_t)tail[1];
    if (ws.path_used == GM_PATH_TC && ctx->schedule != 1 && tail[4] > 0) {   // persistent tcgen05 grid
        const unsigned long long t0 = ~tail[2], first = ~tail[3], last = tail[4];
        if (last > t0) S.cta_finish_spread = (float)((double)(last - first) / (double)(last - t0));
    }
    cudaEventElapsedTime(&S.ms_device, ws.ev[0], ws.ev[3]);
    cudaEventElapsedTime(&S.ms_match, ws.ev[1], ws.ev[2]);
    S.path_used = ws.path_used;
    S.kernel_launches = ws.launches;
    (void)ctx;
}

}  // namespace gm

// ================================================================================================ C ABI
extern "C" {

gm_status gm_create(const gm_config *cfg, gm_ctx **out)
{
    if (!cfg || !out) return fail(GM_ERR_INVALID, "gm_create: null argument");
    *out = nullptr;
    if (cfg->path < GM_PATH_AUTO || cfg->path > GM_PATH_SIMT) return fail(GM_ERR_INVALID, "gm_create: bad path");
    int cell_shift = 0;   // automatic unless configured
    if (cfg->cell_px) {
        int c = cfg->cell_px, sh = 0;
        while ((1 << sh) < c) ++sh;
        if ((1 << sh) != c || sh < kMinCellShift || sh > kMaxCellShift)
            return fail(GM_ERR_INVALID, "gm_create: cell_px must be a power of two in [4, 128]");
        cell_shift = sh;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return fail(GM_ERR_CUDA, "gm_create: CUDA device %d unavailable", cfg->device);
    }
    GM_CUDA(cudaSetDevice(cfg->device));
    gm_ctx *ctx = new gm_ctx();
    ctx->device = cfg->device;
    ctx->budget = cfg->mem_budget_bytes;
    ctx->path = cfg->path;
    ctx->cell_shift = cell_shift;
    ctx->max_inflight = cfg->max_inflight > 0 ? cfg->max_inflight : 2;
    if (cfg->tuner_cache) ctx->tuner_cache = cfg->tuner_cache;
    if (cfg->cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return fail(GM_ERR_CUDA, "gm_create: cudaStreamCreate failed");
        }
        ctx->own_stream = true;
    }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, cfg->device);
    noalloc_setup(cfg->device);   // gm_band_candidates_static's scratch array: loaded here, not in that call
    if (workspace_init(ctx->ws, ctx->stream) != GM_OK || workspace_init(ctx->ws2, ctx->ws.stream) != GM_OK ||
        cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_stage, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_desc, cudaEventDisableTiming) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        workspace_free(ctx, ctx->ws2);   // whatever was created: events and streams (no buffers yet)
        workspace_free(ctx, ctx->ws);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        if (ctx->ev_stage) cudaEventDestroy(ctx->ev_stage);
        if (ctx->ev_desc) cudaEventDestroy(ctx->ev_desc);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return fail(GM_ERR_CUDA, "gm_create: stream or event creation failed: %s", cudaGetErrorString(e));
    }
    *out = ctx;
    return GM_OK;
}

gm_status gm_destroy(gm_ctx *ctx)
{
    if (!ctx) return fail(GM_ERR_INVALID, "gm_destroy: null context");
    cudaSetDevice(ctx->device);
    if (ctx->server) {
        server_stop(ctx->server);
        ctx->server = nullptr;
    }
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    for (auto &kv : ctx->images) {
        release_block(kv.second);
        delete kv.second;
    }
    ctx->images.clear();
    for (auto &kv : ctx->coarse) free_dev(ctx, kv.second.lists);
    ctx->coarse.clear();
    workspace_free(ctx, ctx->ws2);   // shares ws's stream: freed first
    workspace_free(ctx, ctx->ws);
    for (DevBuf *b : {&ctx->d_imgs, &ctx->d_maps, &ctx->d_stage, &ctx->d_work, &ctx->d_bad, &ctx->d_bitmap, &ctx->d_tune,
                      &ctx->d_btab, &ctx->d_pairs, &ctx->d_pairs_out, &ctx->d_pairs_pool, &ctx->d_tracks, &ctx->d_tri,
                      &ctx->d_tri_out, &ctx->d_coarse_tab, &ctx->d_coarse_stage, &ctx->d_coarse_out, &ctx->d_approx, &ctx->d_segs,
                      &ctx->d_selftest})
        free_dev(ctx, *b);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->ev_stage) cudaEventDestroy(ctx->ev_stage);
    if (ctx->ev_desc) cudaEventDestroy(ctx->ev_desc);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return GM_OK;
}

gm_status gm_set_option(gm_ctx *ctx, int32_t key, int64_t value)
{
    if (!ctx) return fail(GM_ERR_INVALID, "gm_set_option: null context");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    switch (key) {
    case GM_OPT_PATH:
        if (value < GM_PATH_AUTO || value > GM_PATH_SIMT) return fail(GM_ERR_INVALID, "bad path %lld", (long long)value);
        ctx->path = (int32_t)value;
        return GM_OK;
    case GM_OPT_SCHEDULE:
        if (value < 0 || value > 1) return fail(GM_ERR_INVALID, "bad schedule %lld", (long long)value);
        ctx->schedule = (int32_t)value;
        return GM_OK;
    case GM_OPT_CELL_PX: {
        if (value == 0) {   // automatic
            ctx->cell_shift = 0;
            return GM_OK;
        }
        int sh = 0;
        while ((1ll << sh) < value) ++sh;
        if ((1ll << sh) != value || sh < kMinCellShift || sh > kMaxCellShift)
            return fail(GM_ERR_INVALID, "cell_px must be a power of two in [4, 128]");
        ctx->cell_shift = sh;
        return GM_OK;
    }
    case GM_OPT_MMA_GROUP:
        if (value != 16 && value != 32) return fail(GM_ERR_INVALID, "mma group must be 16 or 32 queries");
        ctx->mma_mt = (int32_t)(value / 16);
        return GM_OK;
    case GM_OPT_STREAM_CAP:
        if (value < 1 || value > (int64_t)1 << 34) return fail(GM_ERR_INVALID, "bad stream capacity");
        ctx->ws.stream_cap = value;
        free_dev(ctx, ctx->ws.d_stream);
        return GM_OK;
    case GM_OPT_GRAPH:
        if (value < 0 || value > 1) return fail(GM_ERR_INVALID, "bad graph flag");
        ctx->graph = (int32_t)value;
        return GM_OK;
    case GM_OPT_EVICT_LRU:
        if (value < 0 || value > 1) return fail(GM_ERR_INVALID, "bad eviction flag");
        ctx->evict_lru = (int32_t)value;
        return GM_OK;
    case GM_OPT_TC_PIPE:
        if (value < 0 || value >= kTcPipes) return fail(GM_ERR_INVALID, "tc pipeline geometry must be 0, 1 or 2");
        ctx->tc_pipe = (int32_t)value;
        return GM_OK;
    default:
        return fail(GM_ERR_INVALID, "unknown option %d", key);
    }
}

}  // extern "C"

namespace gm {
namespace {

// Layout of one resident image block: xy, perm, inv_perm, desc, norm, col_off, xy_r, idx_r, row_off, desc_h, scale,
// norm256, rec, ext_h (256-byte aligned arrays).
struct ImageLayout {
    int sh = 0, gx = 0, gy = 0;
    int64_t m = 0;
    size_t offs[14] = {};
    size_t tot = 0;
};

ImageLayout image_layout(const gm_ctx *ctx, int32_t width, int32_t height, int32_t n)
{
    ImageLayout L;
    // grid cell: the configured size, or automatically 4 px unless the image is so large that the grid would cross
    // more lines than the tcgen05 kernel's run table holds
    L.sh = ctx->cell_shift;
    if (L.sh == 0) {
        L.sh = kMinCellShift;
        while (L.sh < kMaxCellShift && ((std::max(width, height) + (1 << L.sh) - 1) >> L.sh) > match_tc_max_grid_lines())
            ++L.sh;
    }
    const int cs = 1 << L.sh;
    L.gx = (width + cs - 1) / cs;
    L.gy = (height + cs - 1) / cs;
    L.m = (int64_t)L.gx * L.gy;
    const size_t N = (size_t)n;
    const size_t sz[14] = {8 * N, 4 * N, 4 * N, 128 * N, 4 * N, 4 * (size_t)(L.m + 2), 8 * N, 4 * N,
                           4 * (size_t)(L.m + 2), 256 * N, 4 * N, 4 * N, 16 * (N + 1), 32 * N};
    for (int k = 0; k < 14; ++k) {
        L.offs[k] = L.tot;
        L.tot += align_up(std::max<size_t>(sz[k], 1), 256);
    }
    return L;
}

ImageDev image_dev(const ImageLayout &L, void *block, int32_t width, int32_t height, int32_t n)
{
    char *bp = static_cast<char *>(block);
    ImageDev dev{};
    dev.n = n; dev.width = width; dev.height = height; dev.cell_shift = L.sh; dev.gx = L.gx; dev.gy = L.gy;
    dev.xy = reinterpret_cast<float2 *>(bp + L.offs[0]);
    dev.perm = reinterpret_cast<int32_t *>(bp + L.offs[1]);
    dev.inv_perm = reinterpret_cast<int32_t *>(bp + L.offs[2]);
    dev.desc = reinterpret_cast<int8_t *>(bp + L.offs[3]);
    dev.norm = reinterpret_cast<int32_t *>(bp + L.offs[4]);
    dev.col_off = reinterpret_cast<int32_t *>(bp + L.offs[5]);
    dev.xy_r = reinterpret_cast<float2 *>(bp + L.offs[6]);
    dev.idx_r = reinterpret_cast<int32_t *>(bp + L.offs[7]);
    dev.row_off = reinterpret_cast<int32_t *>(bp + L.offs[8]);
    dev.desc_h = reinterpret_cast<uint16_t *>(bp + L.offs[9]);
    dev.norm256 = reinterpret_cast<int32_t *>(bp + L.offs[11]);
    dev.rec = reinterpret_cast<int4 *>(bp + L.offs[12]);
    dev.ext_h = reinterpret_cast<uint16_t *>(bp + L.offs[13]);
    return dev;
}

// Grows a per-slot device table (image records or TMA descriptors) to `need` bytes, keeping its contents.
gm_status grow_table(gm_ctx *ctx, DevBuf &t, size_t need, size_t min_bytes, cudaStream_t s, const char *what)
{
    if (t.bytes >= need) return GM_OK;
    DevBuf nb;
    const size_t cap = align_up(std::max(need * 2, min_bytes), 256);
    if (cudaMalloc(&nb.p, cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(GM_ERR_NOMEM, "image registration: %s table allocation failed", what);
    }
    nb.bytes = cap;
    if (t.p) {
        cudaMemcpyAsync(nb.p, t.p, t.bytes, cudaMemcpyDeviceToDevice, s);
        cudaStreamSynchronize(s);
    }
    free_dev(ctx, t);
    t = nb;
    ctx->bytes_work += cap;
    return GM_OK;
}

// Runs the batched counting sort over images [k0, k1): with `build` false only the counts and the per-image
// out-of-image keypoint counts (bad + k0 ...), with `build` true the whole sort into the images' blocks.  Images
// are taken in sub-batches so that the shared work arrays stay bounded.
gm_status bucket_batches(gm_ctx *ctx, int32_t count, const gm_image *imgs, const std::vector<ImageLayout> &L,
                         const std::vector<const float2 *> &raw_xy, const std::vector<const uint8_t *> &raw_desc,
                         const std::vector<ImageDev> *dev, unsigned long long *d_bad, cudaStream_t s)
{
    constexpr int64_t kMaxS = int64_t(1) << 24;   // count entries per sub-batch
    constexpr int32_t kMaxK = 4096;
    int32_t k0 = 0;
    while (k0 < count) {
        int32_t k1 = k0;
        int64_t S = 0;
        while (k1 < count && k1 - k0 < kMaxK && (k1 == k0 || S + 2 * (L[k1].m + 2) <= kMaxS)) {
            S += 2 * (L[k1].m + 2);
            ++k1;
        }
        const int32_t K = k1 - k0;
        // host table: jobs, kp_prefix, cnt_prefix, rec_prefix
        const size_t jobs_b = align_up(sizeof(BucketJob) * K, 256), pre_b = align_up(sizeof(int64_t) * (K + 1), 256);
        std::vector<char> tab(jobs_b + 3 * pre_b);
        BucketJob *J = reinterpret_cast<BucketJob *>(tab.data());
        int64_t *kp = reinterpret_cast<int64_t *>(tab.data() + jobs_b);
        int64_t *cp = reinterpret_cast<int64_t *>(tab.data() + jobs_b + pre_b);
        int64_t *rp = reinterpret_cast<int64_t *>(tab.data() + jobs_b + 2 * pre_b);
        int64_t nk = 0, ck = 0;
        for (int32_t k = 0; k < K; ++k) {
            const gm_image &g = imgs[k0 + k];
            const ImageLayout &l = L[k0 + k];
            BucketJob j{};
            j.xy_raw = raw_xy[k0 + k];
            j.desc_raw = raw_desc[k0 + k];
            j.n = g.n; j.width = g.width; j.height = g.height; j.cell_shift = l.sh; j.gx = l.gx; j.gy = l.gy;
            j.m = (int32_t)(l.m + 1);   // the cells and the out-of-image cell
            j.kp_base = nk;
            j.cnt_base = ck;
            if (dev) {
                const ImageDev &d = (*dev)[k0 + k];
                j.xy = const_cast<float2 *>(d.xy); j.xy_r = const_cast<float2 *>(d.xy_r);
                j.perm = const_cast<int32_t *>(d.perm); j.inv_perm = const_cast<int32_t *>(d.inv_perm);
                j.norm = const_cast<int32_t *>(d.norm); j.norm256 = const_cast<int32_t *>(d.norm256);
                j.col_off = const_cast<int32_t *>(d.col_off); j.row_off = const_cast<int32_t *>(d.row_off);
                j.idx_r = const_cast<int32_t *>(d.idx_r); j.desc = const_cast<int8_t *>(d.desc);
                j.desc_h = const_cast<uint16_t *>(d.desc_h); j.rec = const_cast<int4 *>(d.rec);
                j.ext_h = const_cast<uint16_t *>(d.ext_h);
            }
            J[k] = j;
            kp[k] = nk;
            cp[k] = ck;
            rp[k] = nk + k;
            nk += g.n;
            ck += 2 * ((int64_t)j.m + 1);
        }
        kp[K] = nk;
        cp[K] = ck;
        rp[K] = nk + K;
        gm_status st;
        if ((st = ensure_dev(ctx, ctx->d_btab, tab.size())) != GM_OK) return st;
        const size_t work_ints = (size_t)ck + (size_t)ck + 1 + (size_t)ck / 1024 + 8;
        if ((st = ensure_dev(ctx, ctx->d_work, sizeof(int32_t) * work_ints)) != GM_OK) return st;
        GM_CUDA(cudaMemcpyAsync(ctx->d_btab.p, tab.data(), tab.size(), cudaMemcpyHostToDevice, s));
        char *dt = static_cast<char *>(ctx->d_btab.p);
        const BucketJob *dJ = reinterpret_cast<const BucketJob *>(dt);
        const int64_t *dkp = reinterpret_cast<const int64_t *>(dt + jobs_b);
        const int64_t *dcp = reinterpret_cast<const int64_t *>(dt + jobs_b + pre_b);
        const int64_t *drp = reinterpret_cast<const int64_t *>(dt + jobs_b + 2 * pre_b);
        int32_t *work = static_cast<int32_t *>(ctx->d_work.p);
        GM_CUDA(launch_bucket_batch_count(dJ, dkp, K, nk, work, ck, d_bad + k0, s));
        if (dev) GM_CUDA(launch_bucket_batch_build(dJ, dkp, dcp, drp, K, nk, work, ck, work + ck, work + 2 * ck + 1, s));
        // the next sub-batch's table and work arrays are written in stream order, after the kernels above (a
        // reallocation goes through cudaFree, which waits for the device)
        k0 = k1;
    }
    return GM_OK;
}

}  // namespace

int64_t user_image_bytes(gm_ctx *ctx, int32_t id);
int64_t evict_user_image(gm_ctx *ctx, int32_t id);

namespace {

// Caller images that may be evicted for this call: not among the images being put, and not referenced by a serving
// request that has not finished.
std::vector<int32_t> evictable(gm_ctx *ctx, const gm_image *imgs, int32_t count)
{
    std::unordered_set<int32_t> keep;
    for (int32_t k = 0; k < count; ++k) keep.insert(imgs[k].image_id);
    if (ctx->server) server_referenced(ctx->server, keep);
    std::vector<int32_t> ids;
    for (auto &kv : ctx->images)
        if (kv.first >= 0 && kv.second->pins == 0 && !keep.count(kv.first)) ids.push_back(kv.first);
    return ids;
}

// Bytes that evicting every evictable image (with its coarse views) would free.
int64_t evictable_bytes(gm_ctx *ctx, const gm_image *imgs, int32_t count)
{
    int64_t b = 0;
    for (int32_t id : evictable(ctx, imgs, count)) b += user_image_bytes(ctx, id);
    return b;
}

// Evicts evictable images, least recently used first, until `need` bytes are free.
void evict_lru_images(gm_ctx *ctx, const gm_image *imgs, int32_t count, int64_t need)
{
    std::vector<std::pair<uint64_t, int32_t>> order;
    for (int32_t id : evictable(ctx, imgs, count)) order.push_back({ctx->images.at(id)->last_use, id});
    std::sort(order.begin(), order.end());
    for (size_t k = 0; k < order.size() && need > 0; ++k) {
        need -= evict_user_image(ctx, order[k].second);
        ++ctx->images_evicted;
    }
}

}  // namespace

// All inputs are validated before anything registered changes; the device work of all images is enqueued back to
// back with two stream synchronisations in total (after the keypoint check, and at the end).
gm_status put_images(gm_ctx *ctx, int32_t count, const gm_image *imgs, int32_t on_device, const char *fn,
                     bool internal)
{
    gm::NvtxRange nvtx_(fn);
    if (!ctx) return fail(GM_ERR_INVALID, "%s: null context", fn);
    if (count < 0 || (count > 0 && !imgs) || (on_device != 0 && on_device != 1))
        return fail(GM_ERR_INVALID, "%s: bad arguments", fn);
    for (int32_t k = 0; k < count; ++k) {
        const gm_image &g = imgs[k];
        if ((g.image_id < 0) != internal || g.width <= 0 || g.height <= 0 || g.width > (1 << 20) || g.height > (1 << 20) || g.n < 0 ||
            (g.n > 0 && (!g.xy || !g.desc)))
            return fail(GM_ERR_INVALID, "%s: bad arguments (id %d, %dx%d, n %d)", fn, g.image_id, g.width, g.height, g.n);
        for (int32_t l = 0; l < k; ++l)
            if (imgs[l].image_id == g.image_id) return fail(GM_ERR_INVALID, "%s: image id %d given twice", fn, g.image_id);
    }
    if (count == 0) return GM_OK;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA(cudaSetDevice(ctx->device));
    std::vector<ImageLayout> L(count);
    // page-locked inputs are read by the binning kernels in place (one pass over the link, no staging copy)
    std::vector<const void *> in_xy(count, nullptr), in_desc(count, nullptr);
    size_t stage_bytes = 0, new_bytes = 0, replaced = 0;
    for (int32_t k = 0; k < count; ++k) {
        const gm_image &g = imgs[k];
        L[k] = image_layout(ctx, g.width, g.height, g.n);
        if (L[k].m + 2 > INT32_MAX / 4) return fail(GM_ERR_INVALID, "%s: grid too large (image %d)", fn, g.image_id);
        if (on_device && g.n > 0 &&
            ((reinterpret_cast<uintptr_t>(g.xy) & 7) != 0 || (reinterpret_cast<uintptr_t>(g.desc) & 15) != 0))
            return fail(GM_ERR_INVALID, "%s: image %d: device xy must be 8-byte and desc 16-byte aligned", fn,
                        g.image_id);
        if (!on_device && g.n > 0) {
            const void *mxy = mapped_host_ptr(g.xy), *mds = mxy ? mapped_host_ptr(g.desc) : nullptr;
            if (mxy && mds && (reinterpret_cast<uintptr_t>(mxy) & 7) == 0 && (reinterpret_cast<uintptr_t>(mds) & 15) == 0) {
                in_xy[k] = mxy;
                in_desc[k] = mds;
            } else {
                stage_bytes += align_up(8 * (size_t)g.n + 1, 256) + align_up(128 * (size_t)g.n + 1, 256);
            }
        }
        auto it = ctx->images.find(g.image_id);
        const bool reuse = it != ctx->images.end() && it->second->bytes >= L[k].tot;
        if (!reuse) {
            new_bytes += L[k].tot;
            if (it != ctx->images.end()) replaced += it->second->bytes;
        }
    }
    int64_t over = ctx->budget ? (int64_t)(ctx->bytes_images - replaced + new_bytes + ctx->bytes_work) -
                                     (int64_t)ctx->budget
                               : 0;
    if (over > 0) {   // without eviction, or when evicting every other image would not make room: refuse now
        if (!ctx->evict_lru || internal || evictable_bytes(ctx, imgs, count) < over)
            return fail(GM_ERR_BUDGET, "%s: %zu bytes of images exceed the device-memory budget", fn, new_bytes);
    }
    cudaStream_t s = ctx->ws.stream;
    gm_status st;
    // 1. stage host inputs and check every keypoint (nothing registered is touched yet)
    std::vector<const float2 *> raw_xy(count);
    std::vector<const uint8_t *> raw_desc(count);
    if (stage_bytes && (st = ensure_dev(ctx, ctx->d_stage, stage_bytes + 256)) != GM_OK) return st;
    // coordinates go up on the stream (the keypoint check needs them); descriptors on the copy stream, so that their
    // upload overlaps the check and is waited for only before the descriptors are binned
    const bool side = stage_bytes && ctx->copy_stream;
    if (side) {
        // the staging area is free once earlier work on s and an earlier call's uploads (even one that failed before
        // its binning) are done
        GM_CUDA(cudaStreamWaitEvent(s, ctx->ev_desc, 0));
        GM_CUDA(cudaEventRecord(ctx->ev_stage, s));
        GM_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_stage, 0));
    }
    {
        char *sp = static_cast<char *>(ctx->d_stage.p);
        for (int32_t k = 0; k < count; ++k) {
            const gm_image &g = imgs[k];
            raw_xy[k] = reinterpret_cast<const float2 *>(g.xy);
            raw_desc[k] = g.desc;
            if (on_device || g.n == 0) continue;
            if (in_xy[k]) {
                raw_xy[k] = static_cast<const float2 *>(in_xy[k]);
                raw_desc[k] = static_cast<const uint8_t *>(in_desc[k]);
                continue;
            }
            const size_t N = (size_t)g.n, xy_al = align_up(8 * N + 1, 256);
            GM_CUDA(cudaMemcpyAsync(sp, g.xy, 8 * N, cudaMemcpyHostToDevice, s));
            GM_CUDA(cudaMemcpyAsync(sp + xy_al, g.desc, 128 * N, cudaMemcpyHostToDevice, side ? ctx->copy_stream : s));
            raw_xy[k] = reinterpret_cast<const float2 *>(sp);
            raw_desc[k] = reinterpret_cast<const uint8_t *>(sp + xy_al);
            sp += xy_al + align_up(128 * N + 1, 256);
        }
    }
    if (side) GM_CUDA(cudaEventRecord(ctx->ev_desc, ctx->copy_stream));
    if ((st = ensure_dev(ctx, ctx->d_bad, sizeof(unsigned long long) * (size_t)count)) != GM_OK) return st;
    unsigned long long *d_bad = static_cast<unsigned long long *>(ctx->d_bad.p);
    if ((st = bucket_batches(ctx, count, imgs, L, raw_xy, raw_desc, nullptr, d_bad, s)) != GM_OK) return st;
    std::vector<unsigned long long> bad(count);
    GM_CUDA(cudaMemcpyAsync(bad.data(), d_bad, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, s));
    GM_CUDA(cudaStreamSynchronize(s));
    // everything later on s (the binning of the descriptors, or the next call's staging) comes after the upload
    if (side) GM_CUDA(cudaStreamWaitEvent(s, ctx->ev_desc, 0));
    for (int32_t k = 0; k < count; ++k)
        if (bad[k])
            return fail(GM_ERR_INVALID, "%s: image %d: %llu keypoints outside [0,%d)x[0,%d)", fn, imgs[k].image_id,
                        bad[k], imgs[k].width, imgs[k].height);
    // 2. destination blocks: a replaced image's block when it is large enough (no serving batch may still read it)
    if (ctx->server) server_drain(ctx->server);
    if (over > 0) evict_lru_images(ctx, imgs, count, over);   // the inputs are valid and nothing reads the images
    // every new block of the call comes out of one allocation (one cudaMalloc instead of one per image)
    std::vector<void *> block(count, nullptr);
    std::vector<char> fresh(count, 0);
    std::vector<size_t> slab_off(count, 0);
    size_t slab_bytes = 0;
    for (int32_t k = 0; k < count; ++k) {
        auto it = ctx->images.find(imgs[k].image_id);
        if (it != ctx->images.end() && it->second->bytes >= L[k].tot) {
            block[k] = it->second->block;
        } else {
            fresh[k] = 1;
            slab_off[k] = slab_bytes;
            slab_bytes += align_up(L[k].tot, 256);
        }
    }
    Slab *slab = nullptr;
    if (slab_bytes) {
        void *p = nullptr;
        if (cudaMalloc(&p, slab_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(GM_ERR_NOMEM, "%s: cudaMalloc of %zu bytes failed", fn, slab_bytes);
        }
        slab = new Slab{p, 0};
        for (int32_t k = 0; k < count; ++k)
            if (fresh[k]) block[k] = static_cast<char *>(p) + slab_off[k];
    }
    // 3. bin every image into its block (the counts are recomputed: the work arrays hold one sub-batch)
    std::vector<ImageDev> dev(count);
    for (int32_t k = 0; k < count; ++k) dev[k] = image_dev(L[k], block[k], imgs[k].width, imgs[k].height, imgs[k].n);
    st = bucket_batches(ctx, count, imgs, L, raw_xy, raw_desc, &dev, d_bad, s);
    cudaError_t e = cudaSuccess;
    std::vector<CopySeg> segs;   // scales read in place from page-locked memory, all in one launch
    for (int32_t k = 0; k < count && st == GM_OK && e == cudaSuccess; ++k)
        if (imgs[k].n > 0 && imgs[k].scale) {
            char *dst = static_cast<char *>(block[k]) + L[k].offs[10];
            const void *msc = on_device ? nullptr : mapped_host_ptr(imgs[k].scale);
            if (msc && (reinterpret_cast<uintptr_t>(msc) & 3) == 0)
                segs.push_back(CopySeg{msc, dst, (int64_t)imgs[k].n});
            else
                e = cudaMemcpyAsync(dst, imgs[k].scale, 4 * (size_t)imgs[k].n,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        }
    if (st == GM_OK && e == cudaSuccess && !segs.empty()) {
        if ((st = ensure_dev(ctx, ctx->d_segs, sizeof(CopySeg) * segs.size())) == GM_OK) {
            e = cudaMemcpyAsync(ctx->d_segs.p, segs.data(), sizeof(CopySeg) * segs.size(), cudaMemcpyHostToDevice, s);
            for (size_t j0 = 0; j0 < segs.size() && e == cudaSuccess; j0 += 65535) {
                const dim3 grid(8, (unsigned)std::min<size_t>(segs.size() - j0, 65535));
                copy_segments_kernel<<<grid, 256, 0, s>>>(static_cast<const CopySeg *>(ctx->d_segs.p) + j0);
                e = cudaGetLastError();
            }
        }
    }
    // 4. what can still fail comes before the install, so that a failed call leaves every registered image as it
    // was: the slots of new images, the device tables grown to hold them (old entries kept) and the TMA descriptors
    // of each image (tcgen05 path)
    std::vector<int32_t> slot_of(count, -1);
    size_t n_slots = ctx->slots.size();
    {
        size_t q = 0;
        for (int32_t k = 0; k < count; ++k) {
            if (ctx->images.count(imgs[k].image_id)) continue;
            while (q < ctx->slots.size() && ctx->slots[q]) ++q;
            slot_of[k] = (int32_t)(q < ctx->slots.size() ? q++ : n_slots++);
        }
    }
    if (st == GM_OK && e == cudaSuccess)
        st = grow_table(ctx, ctx->d_imgs, sizeof(ImageDev) * n_slots, 4096, s, "image");
    if (st == GM_OK && e == cudaSuccess)
        st = grow_table(ctx, ctx->d_maps, sizeof(TmaMaps) * n_slots, sizeof(TmaMaps) * 16, s, "TMA descriptor");
    // the TMA descriptors depend only on the descriptor rows, the records and n: a re-put into the same block with
    // as many keypoints keeps them
    std::vector<TmaMaps> maps(count);
    std::vector<char> same_maps(count, 0);
    for (int32_t k = 0; k < count && st == GM_OK && e == cudaSuccess; ++k) {
        auto it = ctx->images.find(imgs[k].image_id);
        const ImageDev *old = it != ctx->images.end() ? &it->second->dev : nullptr;
        same_maps[k] = imgs[k].n > 0 && old && old->n == dev[k].n && old->desc_h == dev[k].desc_h &&
                       old->rec == dev[k].rec;
        std::memset(&maps[k], 0, sizeof(TmaMaps));
        if (!same_maps[k] && imgs[k].n > 0) st = encode_maps(dev[k], maps[k]);
    }
    if (st != GM_OK || e != cudaSuccess) {
        cudaStreamSynchronize(s);
        if (slab) {   // no image holds it yet
            cudaFree(slab->p);
            delete slab;
        }
        return st != GM_OK ? st : fail(GM_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    }
    // 5. install: replace, or take the slot chosen above
    if (ctx->slots.size() < n_slots) ctx->slots.resize(n_slots, nullptr);
    for (int32_t k = 0; k < count; ++k) {
        const gm_image &g = imgs[k];
        auto it = ctx->images.find(g.image_id);
        ImageSlot *img = nullptr;
        if (it != ctx->images.end()) {
            img = it->second;
            if (fresh[k]) {
                release_block(img);   // nothing reads the old block: serving was drained, synchronous calls ended
                ctx->bytes_images -= img->bytes;
                img->block = block[k];
                img->slab = slab;
                ++slab->refs;
                img->bytes = L[k].tot;
                ctx->bytes_images += L[k].tot;
            }
        } else {
            img = new ImageSlot();
            img->id = g.image_id;
            img->slot = slot_of[k];
            ctx->slots[img->slot] = img;
            ctx->images[g.image_id] = img;
            img->block = block[k];
            img->slab = slab;
            ++slab->refs;
            img->bytes = L[k].tot;
            ctx->bytes_images += L[k].tot;
        }
        img->dev = dev[k];
        img->gen = ++ctx->image_gen;
        img->last_use = ++ctx->use_tick;
        img->scale = reinterpret_cast<const float *>(static_cast<char *>(img->block) + L[k].offs[10]);
        img->has_scale = g.n > 0 && g.scale != nullptr;
        if (!same_maps[k]) img->maps = maps[k];
    }
    // 6. the device tables' entries: one copy each of every slot's entry
    std::vector<ImageDev> tab_dev;
    std::vector<TmaMaps> tab_maps;
    if (count >= 8) {   // many images: both whole tables in two copies instead of two per image
        tab_dev.assign(ctx->slots.size(), ImageDev{});
        tab_maps.resize(ctx->slots.size());
        std::memset(tab_maps.data(), 0, sizeof(TmaMaps) * tab_maps.size());
        for (size_t q = 0; q < ctx->slots.size(); ++q)
            if (ctx->slots[q]) {
                tab_dev[q] = ctx->slots[q]->dev;
                tab_maps[q] = ctx->slots[q]->maps;
            }
        GM_CUDA(cudaMemcpyAsync(ctx->d_imgs.p, tab_dev.data(), sizeof(ImageDev) * tab_dev.size(), cudaMemcpyHostToDevice,
                                s));
        GM_CUDA(cudaMemcpyAsync(ctx->d_maps.p, tab_maps.data(), sizeof(TmaMaps) * tab_maps.size(),
                                cudaMemcpyHostToDevice, s));
    } else {
        for (int32_t k = 0; k < count; ++k) {
            const ImageSlot *img = ctx->images.at(imgs[k].image_id);
            GM_CUDA(cudaMemcpyAsync(static_cast<ImageDev *>(ctx->d_imgs.p) + img->slot, &img->dev, sizeof(ImageDev),
                                    cudaMemcpyHostToDevice, s));
            GM_CUDA(cudaMemcpyAsync(static_cast<TmaMaps *>(ctx->d_maps.p) + img->slot, &img->maps, sizeof(TmaMaps),
                                    cudaMemcpyHostToDevice, s));
        }
    }
    // the staged inputs and the table entries are read asynchronously: finish before returning
    GM_CUDA(cudaStreamSynchronize(s));
    return GM_OK;
}

void release_block(ImageSlot *img)
{
    if (img->slab && --img->slab->refs == 0) {
        cudaFree(img->slab->p);
        delete img->slab;
    }
    img->slab = nullptr;
    img->block = nullptr;
}

void drop_image(gm_ctx *ctx, int32_t image_id)
{
    auto it = ctx->images.find(image_id);
    if (it == ctx->images.end()) return;
    cudaStreamSynchronize(ctx->ws.stream);
    ImageSlot *img = it->second;
    release_block(img);
    ctx->bytes_images -= img->bytes;
    ctx->slots[img->slot] = nullptr;
    ctx->images.erase(it);
    delete img;
}

// Device bytes of a caller image and of its coarse views.
int64_t user_image_bytes(gm_ctx *ctx, int32_t id)
{
    auto it = ctx->images.find(id);
    if (it == ctx->images.end()) return 0;
    int64_t b = (int64_t)it->second->bytes;
    auto cv = ctx->coarse.find(id);
    if (cv != ctx->coarse.end() && !cv->second.all)
        for (int v = 0; v < 3; ++v) {
            auto iv = cv->second.id[v] < 0 ? ctx->images.find(cv->second.id[v]) : ctx->images.end();
            if (iv != ctx->images.end()) b += (int64_t)iv->second->bytes;
        }
    return b;
}

// Drops a caller image and its coarse views; returns the bytes freed (caller holds ctx->mu, serving drained).
int64_t evict_user_image(gm_ctx *ctx, int32_t id)
{
    const int64_t b = user_image_bytes(ctx, id);
    drop_image(ctx, id);
    auto cv = ctx->coarse.find(id);
    if (cv != ctx->coarse.end()) {
        if (!cv->second.all)
            for (int v = 0; v < 3; ++v)
                if (cv->second.id[v] < 0) drop_image(ctx, cv->second.id[v]);
        free_dev(ctx, cv->second.lists);
        ctx->coarse.erase(cv);
    }
    return b;
}

gm_status run_batch(gm_ctx *ctx, Workspace &ws, int32_t n_pairs, const gm_pair *pairs, bool internal, const char *fn)
{
    gm_status st = engine_plan(ctx, ws, n_pairs, pairs, internal);
    if (st != GM_OK) return st;
    for (int attempt = 0;; ++attempt) {
        if ((st = engine_launch(ctx, ws, nullptr)) != GM_OK) return st;
        GM_CUDA(cudaStreamSynchronize(ws.stream));
        engine_stats(ctx, ws, ctx->stats);
        ctx->stats.n_stream_reruns = attempt;
        if (!ws.overflow) break;
        if (attempt >= 2) return fail(GM_ERR_NOMEM, "%s: candidate stream buffer kept overflowing", fn);
        ws.stream_cap = ws.stream_used + ws.stream_used / 4 + 1024;   // grow to what the batch needed, then rerun
    }
    if (ctx->stats.n_device_errors)
        return fail(GM_ERR_TIMEOUT, "%s: %lld device-side waits ran out", fn, (long long)ctx->stats.n_device_errors);
    return GM_OK;
}

}  // namespace gm

extern "C" {

gm_status gm_image_put(gm_ctx *ctx, int32_t image_id, int32_t width, int32_t height, int32_t n, const float *xy,
                       const float *scale, const uint8_t *desc, int32_t on_device)
{
    const gm_image g{image_id, width, height, n, xy, scale, desc};
    return gm::put_images(ctx, 1, &g, on_device, "gm_image_put");
}

gm_status gm_images_put(gm_ctx *ctx, int32_t count, const gm_image *images, int32_t on_device)
{
    return gm::put_images(ctx, count, images, on_device, "gm_images_put");
}

gm_status gm_image_evict(gm_ctx *ctx, int32_t image_id)
{
    if (!ctx) return fail(GM_ERR_INVALID, "gm_image_evict: null context");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->images.find(image_id);
    if (image_id < 0 || it == ctx->images.end())
        return fail(GM_ERR_NOT_FOUND, "gm_image_evict: image %d not registered", image_id);
    if (ctx->server) server_drain(ctx->server);
    evict_user_image(ctx, image_id);   // the image's coarse-stage views go with it
    return GM_OK;
}

gm_status gm_image_info(gm_ctx *ctx, int32_t image_id, int32_t *n)
{
    if (!ctx) return fail(GM_ERR_INVALID, "gm_image_info: null context");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->images.find(image_id);
    if (image_id < 0 || it == ctx->images.end())
        return fail(GM_ERR_NOT_FOUND, "gm_image_info: image %d not registered", image_id);
    if (n) *n = it->second->dev.n;
    return GM_OK;
}

gm_status gm_image_pin(gm_ctx *ctx, int32_t image_id, int32_t pin)
{
    if (!ctx || (pin != 0 && pin != 1)) return fail(GM_ERR_INVALID, "gm_image_pin: bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    auto it = ctx->images.find(image_id);
    if (image_id < 0 || it == ctx->images.end())
        return fail(GM_ERR_NOT_FOUND, "gm_image_pin: image %d not registered", image_id);
    ImageSlot *img = it->second;
    if (!pin && img->pins == 0) return fail(GM_ERR_INVALID, "gm_image_pin: image %d is not pinned", image_id);
    img->pins += pin ? 1 : -1;
    return GM_OK;
}

gm_status gm_image_cache_stats(gm_ctx *ctx, int64_t *images, int64_t *bytes, int64_t *work_bytes, int64_t *evicted)
{
    if (!ctx) return fail(GM_ERR_INVALID, "gm_image_cache_stats: null context");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    int64_t c = 0;
    for (auto &kv : ctx->images) c += kv.first >= 0;
    if (images) *images = c;
    if (bytes) *bytes = (int64_t)ctx->bytes_images;
    if (work_bytes) *work_bytes = (int64_t)ctx->bytes_work;
    if (evicted) *evicted = ctx->images_evicted;
    return GM_OK;
}

gm_status gm_match_pairs(gm_ctx *ctx, int32_t n_pairs, const gm_pair *pairs, int64_t *pair_off, int32_t *matches,
                         int64_t cap, int64_t *n_written)
{
    gm::NvtxRange nvtx_("gm_match_pairs");
    if (!ctx) return fail(GM_ERR_INVALID, "gm_match_pairs: null context");
    if (n_pairs < 0 || (n_pairs > 0 && !pairs) || !pair_off || !n_written || cap < 0 || (cap > 0 && !matches))
        return fail(GM_ERR_INVALID, "gm_match_pairs: bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA(cudaSetDevice(ctx->device));
    *n_written = 0;
    Workspace &ws = ctx->ws;
    if (n_pairs == 0) {
        if (is_device_ptr(pair_off)) GM_CUDA(cudaMemset(pair_off, 0, sizeof(int64_t)));
        else pair_off[0] = 0;
        ctx->stats = gm_stats{};
        return GM_OK;
    }
    gm_status st = run_batch(ctx, ws, n_pairs, pairs, false, "gm_match_pairs");
    if (st != GM_OK) return st;
    const int64_t *h_off = static_cast<const int64_t *>(ws.h_off.p);
    const int64_t total = h_off[n_pairs];
    *n_written = total;
    cudaStream_t s = ws.stream;
    if (is_device_ptr(pair_off))
        GM_CUDA(cudaMemcpyAsync(pair_off, ws.d_off.p, sizeof(int64_t) * (n_pairs + 1), cudaMemcpyDeviceToDevice, s));
    else
        std::memcpy(pair_off, h_off, sizeof(int64_t) * (n_pairs + 1));
    if (total > cap) {
        GM_CUDA(cudaStreamSynchronize(s));
        return fail(GM_ERR_NOMEM, "gm_match_pairs: %lld matches exceed cap %lld", (long long)total, (long long)cap);
    }
    if (total > 0)
        GM_CUDA(cudaMemcpyAsync(matches, ws.d_rows.p, sizeof(int32_t) * 2 * total, cudaMemcpyDefault, s));
    GM_CUDA(cudaStreamSynchronize(s));
    return GM_OK;
}

gm_status gm_band_candidates(gm_ctx *ctx, const gm_pair *pair, int32_t query_begin, int32_t query_count,
                             int64_t *cand_off, int32_t *cand, int64_t cap, int64_t *n_written)
{
    if (!ctx || !pair || !cand_off || !n_written || query_count < 0 || query_begin < 0 || cap < 0 ||
        (cap > 0 && !cand))
        return fail(GM_ERR_INVALID, "gm_band_candidates: bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    GM_CUDA(cudaSetDevice(ctx->device));
    PairDev pd;
    gm_status st = prepare_pair(ctx, *pair, 0, pd);
    if (st != GM_OK) return st;
    if ((int64_t)query_begin + query_count > pd.n_a)
        return fail(GM_ERR_INVALID, "gm_band_candidates: query range beyond |A| = %d", pd.n_a);
    const int32_t nB = ctx->slots[pd.b]->dev.n;
    const int32_t words = (nB + 31) / 32;
    const size_t bm_bytes = sizeof(uint32_t) * (size_t)std::max(1, words) * std::max(1, query_count);
    if ((st = ensure_dev(ctx, ctx->d_bitmap, bm_bytes)) != GM_OK) return st;
    if ((st = ensure_dev(ctx, ctx->ws.d_tab, 256)) != GM_OK) return st;
    if ((st = ensure_dev(ctx, ctx->ws.d_counts, sizeof(int32_t) * std::max(1, query_count))) != GM_OK) return st;
    if ((st = ensure_dev(ctx, ctx->ws.d_off, sizeof(int64_t) * (query_count + 1))) != GM_OK) return st;
    if ((st = ensure_dev(ctx, ctx->ws.d_ctr, sizeof(BatchCounters) * 64 + 256)) != GM_OK) return st;
    if ((st = ensure_host(ctx->ws.h_off, sizeof(int64_t) * (query_count + 1))) != GM_OK) return st;
    if ((st = ensure_host(ctx->ws.h_tab, sizeof(PairDev))) != GM_OK) return st;
    cudaStream_t s = ctx->ws.stream;
    std::memcpy(ctx->ws.h_tab.p, &pd, sizeof(pd));
    GM_CUDA(cudaMemcpyAsync(ctx->ws.d_tab.p, ctx->ws.h_tab.p, sizeof(pd), cudaMemcpyHostToDevice, s));
    GM_CUDA(cudaMemsetAsync(ctx->d_bitmap.p, 0, bm_bytes, s));
    GM_CUDA(cudaMemsetAsync(ctx->ws.d_ctr.p, 0, sizeof(BatchCounters), s));
    uint32_t *bm = static_cast<uint32_t *>(ctx->d_bitmap.p);
    int64_t *d_off = static_cast<int64_t *>(ctx->ws.d_off.p);
    GM_CUDA(launch_candidates_bitmap(static_cast<const ImageDev *>(ctx->d_imgs.p),
                                     static_cast<const PairDev *>(ctx->ws.d_tab.p), query_begin, query_count, bm, words,
                                     static_cast<BatchCounters *>(ctx->ws.d_ctr.p), s));
    GM_CUDA(launch_bitmap_to_csr_count(bm, query_count, words, static_cast<int32_t *>(ctx->ws.d_counts.p), d_off, s));
    int64_t *h_off = static_cast<int64_t *>(ctx->ws.h_off.p);
    GM_CUDA(cudaMemcpyAsync(h_off, d_off, sizeof(int64_t) * (query_count + 1), cudaMemcpyDeviceToHost, s));
    GM_CUDA(cudaStreamSynchronize(s));
    const int64_t total = h_off[query_count];
    *n_written = total;
    if (is_device_ptr(cand_off))
        GM_CUDA(cudaMemcpyAsync(cand_off, d_off, sizeof(int64_t) * (query_count + 1), cudaMemcpyDeviceToDevice, s));
    else
        std::memcpy(cand_off, h_off, sizeof(int64_t) * (query_count + 1));
    if (total > cap) {
        GM_CUDA(cudaStreamSynchronize(s));
        return fail(GM_ERR_NOMEM, "gm_band_candidates: %lld candidates exceed cap %lld", (long long)total,
                    (long long)cap);
    }
    if (total > 0) {
        int32_t *dst = cand;
        const bool dev = is_device_ptr(cand);
        if (!dev) {
            if ((st = ensure_dev(ctx, ctx->ws.d_rows, sizeof(int32_t) * total)) != GM_OK) return st;
            dst = static_cast<int32_t *>(ctx->ws.d_rows.p);
        }
        GM_CUDA(launch_bitmap_to_csr_fill(bm, query_count, words, d_off, dst, s));
        if (!dev) GM_CUDA(cudaMemcpyAsync(cand, dst, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, s));
    }
    GM_CUDA(cudaStreamSynchronize(s));
    return GM_OK;
}

gm_status gm_get_stats(const gm_ctx *ctx, gm_stats *out)
{
    if (!ctx || !out) return fail(GM_ERR_INVALID, "gm_get_stats: null argument");
    *out = ctx->stats;
    return GM_OK;
}

const char *gm_last_error(const gm_ctx *)
{
    return gm::last_error();
}

gm_status gm_submit(gm_ctx *ctx, const gm_pair *pair, uint64_t *ticket)
{
    if (!ctx || !pair || !ticket) return fail(GM_ERR_INVALID, "gm_submit: null argument");
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        if (!ctx->server) {
            ctx->server = server_start(ctx);
            if (!ctx->server) return fail(GM_ERR_CUDA, "gm_submit: could not start the serving loop");
        }
    }
    return server_submit(ctx->server, *pair, ticket);
}

gm_status gm_get_serving_stats(gm_ctx *ctx, gm_serving_stats *out)
{
    if (!ctx || !out) return fail(GM_ERR_INVALID, "gm_get_serving_stats: null argument");
    *out = gm_serving_stats{};
    if (!ctx->server) return GM_OK;
    return server_stats(ctx->server, out);
}

gm_status gm_serving_drain(gm_ctx *ctx)
{
    if (!ctx) return fail(GM_ERR_INVALID, "gm_serving_drain: null context");
    if (ctx->server) server_wait_idle(ctx->server);
    return GM_OK;
}

gm_status gm_poll(gm_ctx *ctx, uint64_t ticket, int32_t *matches, int64_t cap, int64_t *n, int32_t timeout_ms,
                  double *latency_us)
{
    if (!ctx || !n || cap < 0 || (cap > 0 && !matches)) return fail(GM_ERR_INVALID, "gm_poll: bad arguments");
    if (!ctx->server) return fail(GM_ERR_NOT_FOUND, "gm_poll: unknown ticket %llu", (unsigned long long)ticket);
    return server_poll(ctx->server, ticket, matches, cap, n, timeout_ms, latency_us);
}

}  // extern "C"
