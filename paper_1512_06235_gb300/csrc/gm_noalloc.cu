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
// Set-up: gm_create looks up the array's device address with cudaGetSymbolAddress (with the context's device
// current) and keeps it for that device.  The lookup is what loads the array onto the device: 4 MiB of device
// memory per device, held until the process exits and charged to no context's budget (it is shared by every
// context on the device).  Every gm_create refreshes the address, so a context created after a cudaDeviceReset
// sees the new one.  If the lookup failed at gm_create (for instance because a stream capture was under way), the
// first call of this entry point retries it, and that call may then load the array itself: make it before any
// stream capture.
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

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kPairOff = 0;        // PairDev
constexpr size_t kCtrOff = 256;       // BatchCounters
constexpr size_t kCountsOff = 512;    // int32 [query_count], then the bitmap
static_assert(sizeof(PairDev) <= kCtrOff - kPairOff, "pair record slot");
static_assert(sizeof(BatchCounters) <= kCountsOff - kCtrOff, "counter slot");

// The array's device address per device; nullptr until a lookup succeeds (a failed lookup is retried).
struct ScratchAddr {
    std::mutex mu;
    unsigned char *ptr = nullptr;
};
ScratchAddr g_addr[kMaxDevices];

// Looks the address up with `device` current and stores it; returns the CUDA error of the lookup.
cudaError_t lookup_scratch(int device, unsigned char **out)
{
    ScratchAddr &sa = g_addr[device];
    std::lock_guard<std::mutex> lk(sa.mu);
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, gm_static_scratch);
    if (e == cudaSuccess && p) sa.ptr = static_cast<unsigned char *>(p);
    else cudaGetLastError();   // not sticky: clear it so that the caller's next CUDA call does not see it
    *out = sa.ptr;
    return e;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

#define GM_CUDA_S(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return gm::fail(GM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

// Called by gm_create with the context's device current: loads the scratch array and records its address.  A
// failure is not an error of gm_create (only this entry point needs the array); the entry point retries.
void noalloc_setup(int device)
{
    if (device < 0 || device >= kMaxDevices) return;
    unsigned char *p = nullptr;
    lookup_scratch(device, &p);
}

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
    if (!is_device_ptr_on(cand_off, ctx->device) || (cap > 0 && !is_device_ptr_on(cand, ctx->device)))
        return fail(GM_ERR_INVALID, "gm_band_candidates_static: cand_off and cand must be device memory of device %d",
                    ctx->device);
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

    // the address gm_create looked up; if that lookup failed, retry it now (with the device current)
    unsigned char *scr = nullptr;
    {
        ScratchAddr &sa = g_addr[ctx->device];
        std::lock_guard<std::mutex> lk(sa.mu);
        scr = sa.ptr;
    }
    if (!scr) {
        const cudaError_t e = lookup_scratch(ctx->device, &scr);
        if (e != cudaSuccess || !scr)
            return fail(GM_ERR_CUDA, "gm_band_candidates_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    }
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
