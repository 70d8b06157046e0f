// gm_noalloc.cu -- gm_band_candidates_static: the candidate sets of gm_band_candidates without any allocation.
//
// Who needs it: callers that must not allocate while they run.  Two kinds do:
//   - a process whose device memory is fully committed (the context's budget is taken by resident images, or the
//     rest of the GPU belongs to other work), where the workspace growth of gm_band_candidates would fail;
//   - latency-critical loops, where cudaMalloc / cudaFree (which can synchronise the whole device) and
//     cudaHostAlloc (a page-locking system call) would stall unrelated streams or the host thread.
// This entry point needs nothing beyond the context's resident images: its scratch is one fixed file-scope device
// array, and the caller provides the output buffers in device memory.  It computes exactly what gm_band_candidates
// computes (same kernels: the band walk with the exact FP64 edge decision, bitmap, count, scan, fill).
//
// Set-up: the first call on a device (with that device current) looks up the array's device address with
// cudaGetSymbolAddress, once per device; make that first call before any stream capture begins.
// Concurrency: the scratch is shared by every context on a device, so calls that overlap in time on one device (from
// any thread or context) race on it; the caller serialises them.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "gm_ctx.h"

// Scratch of gm_band_candidates_static: pair record, counters, per-query counts and the candidate bitmap.
static constexpr size_t kStaticScratchBytes = size_t(4) << 20;   // 4 MiB per device
static __device__ __align__(256) unsigned char gm_static_scratch[kStaticScratchBytes];

namespace gm {

bool is_device_ptr(const void *p);

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kPairOff = 0;        // PairDev
constexpr size_t kCtrOff = 256;       // BatchCounters
constexpr size_t kCountsOff = 512;    // int32 [query_count], then the bitmap
static_assert(sizeof(PairDev) <= kCtrOff - kPairOff, "pair record slot");
static_assert(sizeof(BatchCounters) <= kCountsOff - kCtrOff, "counter slot");

struct ScratchAddr {
    std::once_flag once;
    unsigned char *ptr = nullptr;
    cudaError_t err = cudaSuccess;
};
ScratchAddr g_addr[kMaxDevices];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

#define GM_CUDA_S(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return gm::fail(GM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace
}  // namespace gm

extern "C" {

gm_status gm_band_candidates_static(gm_ctx *ctx, const gm_pair *pair, int32_t query_begin, int32_t query_count,
                                    int64_t *cand_off, int32_t *cand, int64_t cap, int64_t *n_written)
{
    using namespace gm;
    if (!ctx || !pair || !cand_off || !n_written || query_count < 0 || query_begin < 0 || cap < 0 ||
        (cap > 0 && !cand))
        return fail(GM_ERR_INVALID, "gm_band_candidates_static: bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return fail(GM_ERR_INVALID, "gm_band_candidates_static: device %d beyond the %d supported", ctx->device,
                    kMaxDevices);
    GM_CUDA_S(cudaSetDevice(ctx->device));
    if (!is_device_ptr(cand_off) || (cap > 0 && !is_device_ptr(cand)))
        return fail(GM_ERR_INVALID, "gm_band_candidates_static: cand_off and cand must be device memory");
    PairDev pd;
    gm_status st = prepare_pair(ctx, *pair, 0, pd);
    if (st != GM_OK) return st;
    if ((int64_t)query_begin + query_count > pd.n_a)
        return fail(GM_ERR_INVALID, "gm_band_candidates_static: query range beyond |A| = %d", pd.n_a);
    const int32_t nB = ctx->slots[pd.b]->dev.n;
    const int32_t words = (nB + 31) / 32;
    const size_t qn = (size_t)(query_count > 0 ? query_count : 1);
    const size_t bm_off = kCountsOff + align256(sizeof(int32_t) * qn);
    const size_t bm_bytes = sizeof(uint32_t) * (size_t)(words > 0 ? words : 1) * qn;
    if (bm_off + bm_bytes > kStaticScratchBytes)
        return fail(GM_ERR_INVALID,
                    "gm_band_candidates_static: %d queries x %d bitmap words need %zu bytes of scratch, more than "
                    "the fixed %zu; split the query range",
                    query_count, words, bm_off + bm_bytes, kStaticScratchBytes);

    // once per device, with the device current: the scratch array's device address
    ScratchAddr &sa = g_addr[ctx->device];
    std::call_once(sa.once, [&] {
        void *p = nullptr;
        sa.err = cudaGetSymbolAddress(&p, gm_static_scratch);
        sa.ptr = static_cast<unsigned char *>(p);
    });
    if (sa.err != cudaSuccess || !sa.ptr)
        return fail(GM_ERR_CUDA, "gm_band_candidates_static: cudaGetSymbolAddress: %s", cudaGetErrorString(sa.err));

    unsigned char *scr = sa.ptr;
    PairDev *d_pair = reinterpret_cast<PairDev *>(scr + kPairOff);
    BatchCounters *d_ctr = reinterpret_cast<BatchCounters *>(scr + kCtrOff);
    int32_t *d_counts = reinterpret_cast<int32_t *>(scr + kCountsOff);
    uint32_t *d_bm = reinterpret_cast<uint32_t *>(scr + bm_off);
    cudaStream_t s = ctx->ws.stream;
    // pd stays alive until the stream is synchronised below; the bitmap and the counters must start at zero
    GM_CUDA_S(cudaMemcpyAsync(d_pair, &pd, sizeof(pd), cudaMemcpyHostToDevice, s));
    GM_CUDA_S(cudaMemsetAsync(d_ctr, 0, sizeof(BatchCounters), s));
    GM_CUDA_S(cudaMemsetAsync(d_bm, 0, bm_bytes, s));
    GM_CUDA_S(launch_candidates_bitmap(static_cast<const ImageDev *>(ctx->d_imgs.p), d_pair, query_begin, query_count,
                                       d_bm, words, d_ctr, s));
    GM_CUDA_S(launch_bitmap_to_csr_count(d_bm, query_count, words, d_counts, cand_off, s));
    int64_t total = 0;
    GM_CUDA_S(cudaMemcpyAsync(&total, cand_off + query_count, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GM_CUDA_S(cudaStreamSynchronize(s));
    *n_written = total;
    if (total > cap)
        return fail(GM_ERR_NOMEM, "gm_band_candidates_static: %lld candidates exceed cap %lld", (long long)total,
                    (long long)cap);
    if (total > 0) GM_CUDA_S(launch_bitmap_to_csr_fill(d_bm, query_count, words, cand_off, cand, s));
    GM_CUDA_S(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // extern "C"
