// gm_order.cu -- per-pair query order from the position of each query's epipolar line (App. A Step 2).
//
// The paper sorts the source features by where their epipolar lines cut the target image and groups lines that
// lie within 2 px so that a group shares one candidate set (Sec. 6.2.2, dual lines).  Here the order is kept and
// the sharing is not: every query still gets its own exact band, but consecutive queries have nearby bands, so a
// group of consecutive queries walks nearly the same cells (cache reuse for the SIMT path, dense tiles for the
// tensor-core paths).
//
// All epipolar lines of a pair pass through the epipole e of B (F^T e = 0).  If e is finite and not far away, the
// key is the angle of the line around e (monotonic along the pencil); if e is at or near infinity the lines are
// (nearly) parallel and the key is their signed offset from the image centre.  Keys are quantised to 4096 bins
// between the pair's min and max key and counting-sorted in shared memory, one block per pair.  The order inside
// a bin is arbitrary: it never changes a result, only which queries run side by side.
#include <cstdint>

#include "gm_internal.h"

namespace gm {
namespace {

constexpr int kBins = 4096;
constexpr int kOrderThreads = 1024;
constexpr int kOrderMinBlocks = 2;   // resident blocks per SM that __launch_bounds__ asks the register allocation for
constexpr int kKeyCache = 16384;   // queries whose keys (then bins) a block keeps in shared memory between passes

struct KeyParams {
    float cx, cy;      // image centre of B
    float ux, uy;      // angle mode: unit vector from the epipole to the centre; parallel mode: reference normal
    int parallel;
};

__device__ __forceinline__ float line_key(const float F[9], float2 p, const KeyParams &kp)
{
    const float a = fmaf(F[0], p.x, fmaf(F[1], p.y, F[2]));
    const float b = fmaf(F[3], p.x, fmaf(F[4], p.y, F[5]));
    const float c = fmaf(F[6], p.x, fmaf(F[7], p.y, F[8]));
    const float n = sqrtf(fmaf(a, a, b * b));
    if (!(n > 0.0f) || !isfinite(n)) return 0.0f;
    if (kp.parallel) {
        const float sgn = fmaf(a, kp.ux, b * kp.uy) >= 0.0f ? 1.0f : -1.0f;
        return sgn * fmaf(a, kp.cx, fmaf(b, kp.cy, c)) / n;
    }
    const float dx = -b, dy = a;                                 // line direction
    float th = atan2f(kp.ux * dy - kp.uy * dx, kp.ux * dx + kp.uy * dy);
    const float hp = 1.57079632679489662f;
    if (th > hp) th -= 2.0f * hp;
    else if (th <= -hp) th += 2.0f * hp;
    return th;
}

__device__ KeyParams key_params(const float F[9], float W, float H)
{
    // epipole: the cross product of two columns of F with the largest norm (F^T e = 0)
    const double c0[3] = {F[0], F[3], F[6]}, c1[3] = {F[1], F[4], F[7]}, c2[3] = {F[2], F[5], F[8]};
    const double *pa[3] = {c0, c0, c1}, *pb[3] = {c1, c2, c2};
    double e[3] = {0, 0, 0}, best = -1.0;
    for (int k = 0; k < 3; ++k) {
        const double *u = pa[k], *v = pb[k];
        const double x = u[1] * v[2] - u[2] * v[1], y = u[2] * v[0] - u[0] * v[2], z = u[0] * v[1] - u[1] * v[0];
        const double nn = x * x + y * y + z * z;
        if (nn > best) { best = nn; e[0] = x; e[1] = y; e[2] = z; }
    }
    KeyParams kp;
    kp.cx = 0.5f * W;
    kp.cy = 0.5f * H;
    const double exy = sqrt(e[0] * e[0] + e[1] * e[1]);
    const double far = 50.0 * ((double)W + (double)H);
    if (exy == 0.0) {                       // degenerate F: any order is fine
        kp.parallel = 1; kp.ux = 0.0f; kp.uy = 1.0f;
    } else if (fabs(e[2]) * far < exy) {    // epipole at or near infinity: parallel lines
        kp.parallel = 1;
        kp.ux = (float)(-e[1] / exy);       // reference normal: perpendicular to the epipole direction
        kp.uy = (float)(e[0] / exy);
    } else {
        kp.parallel = 0;
        const double ex = e[0] / e[2], ey = e[1] / e[2];
        double ux = kp.cx - ex, uy = kp.cy - ey;
        const double un = sqrt(ux * ux + uy * uy);
        if (un > 0.0) { ux /= un; uy /= un; } else { ux = 1.0; uy = 0.0; }
        kp.ux = (float)ux;
        kp.uy = (float)uy;
    }
    return kp;
}

__global__ void __launch_bounds__(kOrderThreads, kOrderMinBlocks) order_kernel(const ImageDev *__restrict__ imgs,
                                                              const PairDev *__restrict__ pairs,
                                                              int32_t *__restrict__ qorder)
{
    __shared__ int32_t hist[kBins];
    extern __shared__ float skey[];   // [kKeyCache]: the key of query s, then its bin (each thread its own entries)
    __shared__ float rmin[32], rmax[32];
    __shared__ KeyParams skp;
    __shared__ float sF[9];
    const PairDev &P = pairs[blockIdx.x];
    const ImageDev &A = imgs[P.a];
    const ImageDev &B = imgs[P.b];
    const int nA = A.n;
    if (threadIdx.x < 9) sF[threadIdx.x] = P.F[threadIdx.x];
    for (int k = threadIdx.x; k < kBins; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    if (threadIdx.x == 0) skp = key_params(sF, (float)B.width, (float)B.height);
    __syncthreads();
    const KeyParams kp = skp;
    float F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = sF[k];

    const bool cached = nA <= kKeyCache;   // otherwise every pass recomputes the keys
    int32_t *sbin = reinterpret_cast<int32_t *>(skey);
    float kmin = INFINITY, kmax = -INFINITY;
    for (int s = threadIdx.x; s < nA; s += blockDim.x) {
        const float key = line_key(F, A.xy[s], kp);
        if (cached) skey[s] = key;
        kmin = fminf(kmin, key);
        kmax = fmaxf(kmax, key);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { rmin[wid] = kmin; rmax[wid] = kmax; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        kmin = lane < nw ? rmin[lane] : INFINITY;
        kmax = lane < nw ? rmax[lane] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if (lane == 0) { rmin[0] = kmin; rmax[0] = kmax; }
    }
    __syncthreads();
    kmin = rmin[0];
    kmax = rmax[0];
    const float span = kmax - kmin;
    const float scale = span > 0.0f && isfinite(span) ? (float)kBins / span : 0.0f;

    for (int s = threadIdx.x; s < nA; s += blockDim.x) {
        const float key = cached ? skey[s] : line_key(F, A.xy[s], kp);
        const int bin = min(kBins - 1, max(0, (int)((key - kmin) * scale)));
        if (cached) sbin[s] = bin;
        atomicAdd(&hist[bin], 1);
    }
    __syncthreads();
    // exclusive scan of the 4096 bins: each thread owns 4 consecutive bins
    {
        const int t = threadIdx.x;
        int v0 = hist[4 * t], v1 = hist[4 * t + 1], v2 = hist[4 * t + 2], v3 = hist[4 * t + 3];
        const int tot = v0 + v1 + v2 + v3;
        int incl = tot;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, s);
            if (lane >= s) incl += u;
        }
        __shared__ int32_t wsum[32];
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, w, s);
                if (lane >= s) w += u;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int base = (wid > 0 ? wsum[wid - 1] : 0) + incl - tot;
        hist[4 * t] = base;
        hist[4 * t + 1] = base + v0;
        hist[4 * t + 2] = base + v0 + v1;
        hist[4 * t + 3] = base + v0 + v1 + v2;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nA; s += blockDim.x) {
        int bin;
        if (cached) {
            bin = sbin[s];
        } else {
            const float key = line_key(F, A.xy[s], kp);
            bin = min(kBins - 1, max(0, (int)((key - kmin) * scale)));
        }
        const int pos = atomicAdd(&hist[bin], 1);
        qorder[P.qoff + pos] = s;
    }
}

}  // namespace

cudaError_t launch_order(const ImageDev *imgs, const PairDev *pairs, int32_t n_pairs, int32_t *qorder,
                         cudaStream_t st)
{
    static_assert(kBins == 4 * kOrderThreads, "scan layout");
    constexpr int smem = (int)sizeof(float) * kKeyCache;
    static const cudaError_t attr = cudaFuncSetAttribute(order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    if (n_pairs > 0) order_kernel<<<n_pairs, kOrderThreads, smem, st>>>(imgs, pairs, qorder);
    return cudaGetLastError();
}

}  // namespace gm
