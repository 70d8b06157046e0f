// gm_selftest.cu -- gm_selftest_wait: the failure path of a bounded device-side wait, exercised on purpose (the
// paper has no counterpart).
//
// Every wait in the library's kernels (mbarrier phases, work queues) gives up after a time limit, records the
// failure in device memory and returns, so that the host turns it into GM_ERR_TIMEOUT and the context stays usable.
// This entry point runs that pattern in isolation: one thread waits for a flag in device memory with a bounded
// spin; the host either sets the flag first (the wait succeeds) or leaves it clear (the wait runs out).
#include <cuda_runtime.h>

#include <cstdint>

#include "gm_ctx.h"

namespace gm {
namespace {

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// status[0] = 0: the flag was seen; 1: the time limit ran out first.  The spin also stops after 2^30 polls.
__global__ void wait_flag_kernel(const volatile int32_t *flag, uint64_t limit_ns, int32_t *status)
{
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (*flag != 0) {
            status[0] = 0;
            return;
        }
        if (globaltimer_ns() - t0 > limit_ns) break;
        __nanosleep(500);
    }
    status[0] = 1;
}

}  // namespace
}  // namespace gm

extern "C" {

gm_status gm_selftest_wait(gm_ctx *ctx, int32_t limit_us, int32_t set_flag)
{
    using namespace gm;
    if (!ctx || limit_us < 1 || limit_us > 1000000 || (set_flag != 0 && set_flag != 1))
        return fail(GM_ERR_INVALID, "gm_selftest_wait: bad arguments");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(GM_ERR_CUDA, "gm_selftest_wait: cudaSetDevice");
    gm_status st = ensure_dev(ctx, ctx->d_selftest, 256);
    if (st != GM_OK) return st;
    cudaStream_t s = ctx->ws.stream;
    int32_t *flag = static_cast<int32_t *>(ctx->d_selftest.p), *status = flag + 32;
    const int32_t init[2] = {set_flag, -1};
    int32_t h_status = -1;
    if (cudaMemcpyAsync(flag, &init[0], sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(status, &init[1], sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(GM_ERR_CUDA, "gm_selftest_wait: cudaMemcpyAsync");
    wait_flag_kernel<<<1, 1, 0, s>>>(flag, (uint64_t)limit_us * 1000ull, status);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h_status, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(GM_ERR_CUDA, "gm_selftest_wait: launch");
    if (h_status == 1) return fail(GM_ERR_TIMEOUT, "gm_selftest_wait: the device-side wait ran out after %d us", limit_us);
    if (h_status != 0) return fail(GM_ERR_CUDA, "gm_selftest_wait: no status written");
    return GM_OK;
}

}  // extern "C"
