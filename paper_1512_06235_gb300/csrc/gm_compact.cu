// gm_compact.cu -- output assembly: per-pair match lists sorted by the query index (App. A Step 4 writes one
// decision per query; this turns them into the caller's CSR), and the candidate-set CSR of gm_band_candidates.
#include <cstdint>

#include "gm_band.cuh"
#include "gm_internal.h"

namespace gm {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int block_exclusive_scan(int v, int &total, int32_t *wsum)
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
    const int r = (wid > 0 ? wsum[wid - 1] : 0) + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads) count_matches_kernel(const PairDev *__restrict__ pairs,
                                                                 const int32_t *__restrict__ match_j,
                                                                 int32_t *__restrict__ counts)
{
    __shared__ int32_t wsum[32];
    const PairDev &P = pairs[blockIdx.x];
    int c = 0;
    for (int i = threadIdx.x; i < P.n_a; i += blockDim.x) c += match_j[P.qoff + i] >= 0;
    int total;
    block_exclusive_scan(c, total, wsum);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// off[0..m]: exclusive scan of counts (int64), off[m] = total.  One block.
__global__ void __launch_bounds__(1024) scan64_kernel(const int32_t *__restrict__ counts, int32_t m,
                                                      int64_t *__restrict__ off)
{
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < m; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int64_t v = i < m ? counts[i] : 0;
        int64_t incl = v;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, incl, s);
            if (lane >= s) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int64_t w = lane < nw ? wsum[lane] : 0;
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const int64_t t = __shfl_up_sync(0xffffffffu, w, s);
                if (lane >= s) w += t;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int64_t before = (wid > 0 ? wsum[wid - 1] : 0) + carry;
        if (i < m) off[i] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[m] = carry;
}

__global__ void __launch_bounds__(kThreads) write_matches_kernel(const PairDev *__restrict__ pairs,
                                                                 const int32_t *__restrict__ match_j,
                                                                 const int64_t *__restrict__ pair_off,
                                                                 int32_t *__restrict__ matches)
{
    __shared__ int32_t wsum[32];
    const PairDev &P = pairs[blockIdx.x];
    int64_t out = pair_off[blockIdx.x];
    for (int base = 0; base < P.n_a; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int j = i < P.n_a ? match_j[P.qoff + i] : -1;
        int total;
        const int r = block_exclusive_scan(j >= 0, total, wsum);
        if (j >= 0) {
            matches[2 * (out + r)] = i;
            matches[2 * (out + r) + 1] = j;
        }
        out += total;
    }
}

// ---- candidate sets (diagnostic output of the band walk) ----

__global__ void __launch_bounds__(256) candidates_bitmap_kernel(const ImageDev *__restrict__ imgs,
                                                                const PairDev *__restrict__ pair, int32_t q_begin,
                                                                int32_t q_count, uint32_t *__restrict__ bitmap,
                                                                int32_t words, BatchCounters *__restrict__ ctr)
{
    const int lane = threadIdx.x & 31;
    const int qi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (qi >= q_count) return;
    const PairDev &P = *pair;
    const ImageDev A = imgs[P.a];
    const ImageDev B = imgs[P.b];
    float F[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) F[t] = P.F[t];
    const int s = A.inv_perm[q_begin + qi];
    const float2 q = A.xy[s];
    const BandLine L = band_line(F, q.x, q.y, P.d, (float)B.width, (float)B.height);
    uint32_t *row = bitmap + (int64_t)qi * words;
    unsigned examined = 0, redecided = 0;
    auto visit = [&](bool valid, bool inb, int pos) {
        if (inb) {
            const int j = B.perm[pos];
            atomicOr(row + (j >> 5), 1u << (j & 31));
        }
    };
    band_walk(B, L, F, q.x, q.y, P.d, visit, examined, redecided);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        examined += __shfl_xor_sync(0xffffffffu, examined, o);
        redecided += __shfl_xor_sync(0xffffffffu, redecided, o);
    }
    if (lane == 0) {
        atomicAdd(&ctr->examined, (unsigned long long)examined);
        atomicAdd(&ctr->redecided, (unsigned long long)redecided);
    }
}

__global__ void bitmap_count_kernel(const uint32_t *__restrict__ bitmap, int32_t q_count, int32_t words,
                                    int32_t *__restrict__ counts)
{
    const int lane = threadIdx.x & 31;
    const int qi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (qi >= q_count) return;
    int c = 0;
    for (int w = lane; w < words; w += 32) c += __popc(bitmap[(int64_t)qi * words + w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) counts[qi] = c;
}

__global__ void bitmap_fill_kernel(const uint32_t *__restrict__ bitmap, int32_t q_count, int32_t words,
                                   const int64_t *__restrict__ off, int32_t *__restrict__ cand)
{
    const int lane = threadIdx.x & 31;
    const int qi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (qi >= q_count) return;
    int64_t out = off[qi];
    for (int base = 0; base < words; base += 32) {
        const int w = base + lane;
        uint32_t bits = w < words ? bitmap[(int64_t)qi * words + w] : 0u;
        const int c = __popc(bits);
        int incl = c;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, s);
            if (lane >= s) incl += t;
        }
        int64_t pos = out + incl - c;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            cand[pos++] = w * 32 + b;
        }
        out += __shfl_sync(0xffffffffu, incl, 31);
    }
}

}  // namespace

cudaError_t launch_count_matches(const PairDev *pairs, int32_t n_pairs, const int32_t *match_j, int32_t *counts,
                                 int64_t *pair_off, cudaStream_t st)
{
    if (n_pairs > 0) count_matches_kernel<<<n_pairs, kThreads, 0, st>>>(pairs, match_j, counts);
    scan64_kernel<<<1, 1024, 0, st>>>(counts, n_pairs, pair_off);
    return cudaGetLastError();
}

cudaError_t launch_write_matches(const PairDev *pairs, int32_t n_pairs, const int32_t *match_j,
                                 const int64_t *pair_off, int32_t *matches, cudaStream_t st)
{
    if (n_pairs > 0) write_matches_kernel<<<n_pairs, kThreads, 0, st>>>(pairs, match_j, pair_off, matches);
    return cudaGetLastError();
}

cudaError_t launch_candidates_bitmap(const ImageDev *imgs, const PairDev *pair, int32_t q_begin, int32_t q_count,
                                     uint32_t *bitmap, int32_t words, BatchCounters *ctr, cudaStream_t st)
{
    if (q_count > 0)
        candidates_bitmap_kernel<<<(q_count + 7) / 8, 256, 0, st>>>(imgs, pair, q_begin, q_count, bitmap, words,
                                                                    ctr);
    return cudaGetLastError();
}

cudaError_t launch_bitmap_to_csr_count(const uint32_t *bitmap, int32_t q_count, int32_t words, int32_t *counts,
                                       int64_t *off, cudaStream_t st)
{
    if (q_count > 0) bitmap_count_kernel<<<(q_count + 7) / 8, 256, 0, st>>>(bitmap, q_count, words, counts);
    scan64_kernel<<<1, 1024, 0, st>>>(counts, q_count, off);
    return cudaGetLastError();
}

cudaError_t launch_bitmap_to_csr_fill(const uint32_t *bitmap, int32_t q_count, int32_t words, const int64_t *off,
                                      int32_t *cand, cudaStream_t st)
{
    if (q_count > 0) bitmap_fill_kernel<<<(q_count + 7) / 8, 256, 0, st>>>(bitmap, q_count, words, off, cand);
    return cudaGetLastError();
}

}  // namespace gm
