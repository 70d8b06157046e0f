// gm_stream.cu -- candidate streams of the query groups of the tensor-core path (App. A Step 3, per group).
//
// For a group of 128 consecutive (line-sorted) queries the union of their bands lies between the two chords of
// the strips' upper and lower envelopes over the walked image axis: the maximum of linear functions is convex and
// lies below the chord between its end values, the minimum is concave and lies above its chord.  Walking the grid
// column by column (or row by row for steep lines), one run of cells per grid line covers every keypoint any query
// of the group can accept; the runs are flattened into a list of column-major keypoint positions (the group's
// candidate stream) in global memory, which the tcgen05 kernel then gathers chunk by chunk.
//
// One warp per group, four groups per block.  Space is reserved with one atomic per block; a stream that would
// overflow the buffer marks its group (the caller grows the buffer and runs the batch again).  Groups that contain
// a whole-image query (d = inf) or an FP64-only line use the whole image and store no stream.
#include <cstdint>

#include "gm_band.cuh"
#include "gm_internal.h"

namespace gm {
namespace {

constexpr int kWarps = 4;
constexpr int kMinBlocks = 1;   // resident blocks per SM that __launch_bounds__ asks the register allocation for
constexpr int kG = kTcQueriesPerItem;   // queries per group
constexpr int kMaxLines = 1024;

__device__ __forceinline__ int pair_of_item(const int64_t *__restrict__ item_off, int n_pairs, int64_t t)
{
    int lo = 0, hi = n_pairs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (item_off[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kWarps * 32, kMinBlocks) stream_kernel(
    const ImageDev *__restrict__ imgs, const PairDev *__restrict__ pairs, const int64_t *__restrict__ item_off,
    int32_t n_pairs, const int32_t *__restrict__ qorder, int64_t item_begin, int64_t item_end,
    GroupDesc *__restrict__ gdesc, int32_t *__restrict__ grows, int32_t *__restrict__ stream, int64_t capacity,
    unsigned long long *__restrict__ used, BatchCounters *__restrict__ ctr, int32_t max_lines)
{
    // per warp: run starts [max_lines] and exclusive run offsets [max_lines + 1] (sized for the batch's images, so
    // that small grids leave room for more resident blocks)
    extern __shared__ int32_t runs_smem[];
    int32_t *const run_start_w = runs_smem + (threadIdx.x >> 5) * (2 * max_lines + 1);
    int32_t *const run_excl_w = run_start_w + max_lines;
    __shared__ int32_t wtotal[kWarps];
    __shared__ unsigned long long wbase[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t item = item_begin + (int64_t)blockIdx.x * kWarps + warp;
    const bool active = item < item_end;
    int total = 0, full = 0, colwise = 1;
    const ImageDev *Bp = nullptr;
    const PairDev *Pp = nullptr;
    const ImageDev *Ap = nullptr;
    if (active) {
        const int pi = pair_of_item(item_off, n_pairs, item);
        const PairDev &P = pairs[pi];
        const ImageDev &A = imgs[P.a];
        const ImageDev &B = imgs[P.b];
        Bp = &B;
        Pp = &P;
        Ap = &A;
        const int q0 = (int)(item - item_off[pi]) * kG;
        const float d = P.d;
        const float W = (float)B.width, H = (float)B.height;
        float F[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) F[t] = P.F[t];
        int s4[kG / 32];
#pragma unroll
        for (int t = 0; t < kG / 32; ++t) {
            const int k = q0 + lane + 32 * t;
            s4[t] = k < P.n_a ? qorder[P.qoff + k] : -1;
            grows[item * kG + lane + 32 * t] = s4[t];
        }
        BandLine L4[kG / 32];
        int votes = 0, nnorm = 0;
#pragma unroll
        for (int t = 0; t < kG / 32; ++t) {
            L4[t].mode = kBandEmpty;
            if (s4[t] >= 0) {
                const float2 q = A.xy[s4[t]];
                L4[t] = band_line(F, q.x, q.y, d, W, H);
                if (L4[t].mode == kBandNormal) { ++nnorm; votes += fabsf(L4[t].b) >= fabsf(L4[t].a); }
                else full = 1;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            votes += __shfl_xor_sync(0xffffffffu, votes, o);
            nnorm += __shfl_xor_sync(0xffffffffu, nnorm, o);
            full |= __shfl_xor_sync(0xffffffffu, full, o);
        }
        colwise = 2 * votes >= nnorm;
        const float ulim = colwise ? W : H, vlim = colwise ? H : W;
        float t0 = -INFINITY, t1 = -INFINITY, b0 = INFINITY, b1 = INFINITY, pad = 0.0f;
#pragma unroll
        for (int t = 0; t < kG / 32; ++t) {
            if (L4[t].mode != kBandNormal) continue;
            float pa = colwise ? L4[t].a : L4[t].b, pb = colwise ? L4[t].b : L4[t].a, c = L4[t].c;
            if (pb < 0.0f) { pa = -pa; pb = -pb; c = -c; }
            const float T = L4[t].t_walk;
            if (!(pb > 1e-30f)) { full = 1; continue; }
            const float ib = 1.0f / pb;
            const float e0 = -c * ib, e1 = -fmaf(pa, ulim, c) * ib, h = T * ib;
            t0 = fmaxf(t0, e0 + h); t1 = fmaxf(t1, e1 + h);
            b0 = fminf(b0, e0 - h); b1 = fminf(b1, e1 - h);
            pad = fmaxf(pad, 8.0f * kU * (fabsf(pa) * ulim + fabsf(c) + T) * ib);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t0 = fmaxf(t0, __shfl_xor_sync(0xffffffffu, t0, o));
            t1 = fmaxf(t1, __shfl_xor_sync(0xffffffffu, t1, o));
            b0 = fminf(b0, __shfl_xor_sync(0xffffffffu, b0, o));
            b1 = fminf(b1, __shfl_xor_sync(0xffffffffu, b1, o));
            pad = fmaxf(pad, __shfl_xor_sync(0xffffffffu, pad, o));
            full |= __shfl_xor_sync(0xffffffffu, full, o);
        }
        pad += 1e-3f + 4.0f * kU * (fabsf(t0) + fabsf(t1) + fabsf(b0) + fabsf(b1));
        const float et0 = t0 + pad, et1 = t1 + pad, eb0 = b0 - pad, eb1 = b1 - pad;
        if (nnorm > 0 && !(isfinite(et0) && isfinite(et1) && isfinite(eb0) && isfinite(eb1))) full = 1;
        const int nlines = colwise ? B.gx : B.gy;
        if (full) {
            total = B.n;
            colwise = 1;
        } else if (nnorm > 0) {
            const float cs = (float)(1 << B.cell_shift), inv_cs = 1.0f / cs;
            const int ng = colwise ? B.gy : B.gx;
            const int32_t *offs = colwise ? B.col_off : B.row_off;
            int carry = 0;
            for (int base_line = 0; base_line < nlines; base_line += 32 * 8) {
                int st[8], en[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int kk = base_line + 32 * t + lane;
                    st[t] = -1;
                    en[t] = 0;
                    if (kk < nlines) {
                        const float u0 = (float)kk * cs, u1 = fminf(u0 + cs, ulim);
                        const float f0 = u0 / ulim, f1 = u1 / ulim;
                        const float top0 = fmaf(et1 - et0, f0, et0), top1 = fmaf(et1 - et0, f1, et0);
                        const float bot0 = fmaf(eb1 - eb0, f0, eb0), bot1 = fmaf(eb1 - eb0, f1, eb0);
                        const float lo = fminf(bot0, bot1), hi = fmaxf(top0, top1);
                        if (hi >= 0.0f && lo < vlim) {
                            const int c0 = max(0, (int)floorf(fmaxf(lo, 0.0f) * inv_cs));
                            const int c1 = min(ng - 1, (int)floorf(fminf(hi, vlim) * inv_cs));
                            if (c0 <= c1) { st[t] = kk * ng + c0; en[t] = kk * ng + c1 + 1; }
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    int s0 = 0, s1 = 0;
                    if (st[t] >= 0) { s0 = offs[st[t]]; s1 = offs[en[t]]; }
                    st[t] = s0;
                    en[t] = s1 - s0;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int kk = base_line + 32 * t + lane;
                    int incl = en[t];
#pragma unroll
                    for (int s = 1; s < 32; s <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, incl, s);
                        if (lane >= s) incl += u;
                    }
                    if (kk < max_lines) {
                        run_start_w[kk] = st[t];
                        run_excl_w[kk] = carry + incl - en[t];
                    }
                    carry += __shfl_sync(0xffffffffu, incl, 31);
                }
            }
            if (lane == 0) run_excl_w[nlines] = carry;
            total = carry;
        }
    }
    // reserve the block's space with one atomic; every stream starts on a 16-byte boundary (reservations are
    // rounded up to four positions) so that the matcher can stage it with 16-byte copies
    if (lane == 0) wtotal[warp] = (active && !full) ? (total + 3) & ~3 : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sum = 0;
        for (int w = 0; w < kWarps; ++w) sum += (unsigned long long)wtotal[w];
        unsigned long long b = sum ? atomicAdd(used, sum) : 0ull;
        for (int w = 0; w < kWarps; ++w) {
            wbase[w] = b;
            b += (unsigned long long)wtotal[w];
        }
    }
    __syncthreads();
    if (!active) return;
    const unsigned long long off = wbase[warp];
    const bool overflow = !full && off + (unsigned long long)((total + 3) & ~3) > (unsigned long long)capacity;
    if (lane == 0) {
        const PairDev &P = *Pp;
        const ImageDev &A = *Ap, &B = *Bp;
        GroupDesc r;
        r.off = (int64_t)off;
        r.a_rec = A.rec;
        r.a_perm = A.perm;
        r.a_desc = A.desc_h;
        r.b_desc = B.desc_h;
        r.b_rec = B.rec;
        r.b_perm = B.perm;
        r.a_slot = P.a;
        r.b_slot = P.b;
        r.a_n = A.n;
        r.b_n = B.n;
        r.total = overflow ? 0 : total;
        r.flags = (full ? 1 : 0) | (overflow ? 2 : 0);
        r.p = P.p;
        r.q = P.q;
        for (int t = 0; t < 9; ++t) r.F[t] = P.F[t];
        r.d = P.d;
        r.W = (float)B.width;
        r.H = (float)B.height;
        r.qoff = P.qoff;
        gdesc[item] = r;
        if (overflow) atomicAdd(&ctr->overflow, 1ull);
        else if (!full && total > kTcStagedPositions) atomicAdd(&ctr->unstaged, 1ull);
        atomicAdd(&ctr->examined, (unsigned long long)total * kG);
    }
    if (full || overflow || total == 0) return;
    // flatten the runs: every lane writes the positions of its grid lines
    const ImageDev &B = *Bp;
    const int nlines = colwise ? B.gx : B.gy;
    for (int kk = lane; kk < nlines; kk += 32) {
        const int e0 = run_excl_w[kk], len = run_excl_w[kk + 1] - e0;
        const int st = run_start_w[kk];
        int32_t *dst = stream + off + e0;
        for (int k = 0; k < len; ++k) dst[k] = colwise ? st + k : B.idx_r[st + k];
    }
}

}  // namespace

cudaError_t launch_stream(const ImageDev *imgs, const PairDev *pairs, const int64_t *item_off, int32_t n_pairs,
                          const int32_t *qorder, int64_t item_begin, int64_t item_end, GroupDesc *gdesc, int32_t *grows,
                          int32_t *stream, int64_t capacity, unsigned long long *used, BatchCounters *ctr,
                          int32_t max_lines, cudaStream_t st)
{
    const int64_t n = item_end - item_begin;
    if (n <= 0) return cudaSuccess;
    if (max_lines < 1 || max_lines > kMaxLines) return cudaErrorInvalidValue;
    static const cudaError_t attr = cudaFuncSetAttribute(stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)(sizeof(int32_t) * kWarps * (2 * kMaxLines + 1)));
    if (attr != cudaSuccess) return attr;
    const size_t smem = sizeof(int32_t) * kWarps * (2 * (size_t)max_lines + 1);
    stream_kernel<<<(unsigned)((n + kWarps - 1) / kWarps), kWarps * 32, smem, st>>>(
        imgs, pairs, item_off, n_pairs, qorder, item_begin, item_end, gdesc, grows, stream, capacity, used, ctr,
        max_lines);
    return cudaGetLastError();
}

}  // namespace gm
