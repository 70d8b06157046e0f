// gm_match_tc.cu -- tcgen05 matching path: warp-specialised pipeline of 128-query x 64-candidate tensor-core tiles.
//
// App. A Steps 3-4 for groups of 128 consecutive queries of one pair (queries sorted by the position of their
// epipolar line, so a group's bands nearly coincide; every query keeps its own exact band).  One persistent CTA
// per SM runs four roles that hand work to each other through mbarriers:
//
//   setup warps (2, alternate groups): the group's FP32 lines and exact-decision thresholds (gm_band.cuh), the
//       chord envelope of the group's strips and one run of cells per grid column (see gm_match_mma.cu for the
//       envelope argument), the run table, and the TMA gather4 of the 128 query descriptors (recentred, fp16:
//       integers in [-128, 127] are exact) into the group's A tile (128-byte-swizzled K-major layout);
//   loader warp: cuts the group's candidate stream into 64-row chunks and gathers, with TMA gather4, the fp16
//       descriptor rows (two K halves) and a 16-byte record per candidate (x, y, |b'|^2 * 256, index) into a
//       4-stage ring; slots past the end of the stream get the image's NaN sentinel record;
//   MMA warp (one elected thread): eight tcgen05.mma.kind::f16 per chunk (M = 128, N = 64, K = 16 each), f32
//       accumulation into one of two tensor-memory buffers.  Products are integers of magnitude <= 2^14 and partial
//       sums <= 2^21 < 2^24, so the accumulator holds the exact integer dot product a'.b';
//   epilogue warps (8 = 4 lane quadrants x 2 column halves): tcgen05.ld of 32 accumulator columns, then per element
//       the exact band test, D = |a'|^2 + |b'|^2 - 2 a'.b' packed with the column into one int32 key, a masked
//       running top-2; at the end of the group the two column halves merge and the integer ratio test
//       q^2 D1 < p^2 D2 decides (Sec. 2.3).
//
// CTA b takes work items b, b + gridDim.x, ... (static order: every role derives the same group sequence).
// Every mbarrier wait gives up after one second; the CTA then raises the batch error counter, every role leaves its
// loop, and the CTA frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "gm_band.cuh"
#include "gm_internal.h"

namespace gm {
namespace {

constexpr int kM = 128;             // queries per group (tensor-memory lanes)
constexpr int kN = 64;              // candidates per chunk
constexpr int kStages = 4;          // candidate chunks in flight
constexpr int kSlots = 2;           // query groups in flight
constexpr int kMaxRuns = 1024;      // grid lines per group walk
constexpr int kEpiWarps = 8;
constexpr int kLoaderWarp = 8, kMmaWarp = 9, kSetupWarp0 = 10;
constexpr int kThreads = 12 * 32;
constexpr int kTmemCols = 2 * kN;   // two accumulator buffers
constexpr int kCounterShards = 64;
constexpr unsigned long long kWaitNs = 1000000000ull;   // one second

constexpr int kAHalf = kM * 128;                    // one K half of a query tile (bytes)
constexpr int kBHalf = kN * 128;                    // one K half of a candidate chunk
constexpr int kOffA = 0;                            // kSlots A tiles
constexpr int kOffB = kOffA + kSlots * 2 * kAHalf;  // kStages candidate chunks
constexpr int kOffRec = kOffB + kStages * 2 * kBHalf;
constexpr int kRecStage = (kN / 4) * 128;         // records of a chunk: one 128-byte slot per quad of 4 records
constexpr int kOffCtl = kOffRec + kStages * kRecStage;
constexpr uint32_t kChunkTx = kN * (256 + 16);      // bytes the loader's TMAs bring per chunk
constexpr uint32_t kATx = kM * 256;

struct Meta {
    int32_t pair, nchunks, total, walk_full, colwise;
};

struct Ctl {
    float ln[kSlots][kM][8];         // a, b, c, thr_lo, thr_hi, qx, qy, walk half-width (or -1 whole image, -2 none)
    int32_t rinfo[kSlots][kM][2];    // original A index (-1: no query), |a'|^2 * 256
    int32_t aidx[kSlots][kM];        // A rows to gather
    int32_t run_start[kSlots][kMaxRuns];
    int32_t run_excl[kSlots][kMaxRuns + 1];
    int32_t merge[kSlots][kM][4];
    Meta meta[kSlots];
    float F[kSlots][9];
    uint64_t stage_full[kStages], stage_empty[kStages], acc_full[2], acc_empty[2];
    uint64_t grp_full[kSlots], grp_empty[kSlots], merge_ready[kSlots];
    uint32_t tmem_base;
    volatile int32_t abort_flag;
    unsigned long long stat[3];
};
constexpr int kSmemBytes = kOffCtl + (int)sizeof(Ctl) + 1024;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase of the given parity; false after one second.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 255) == 0) {
            const uint64_t t = globaltimer();
            if (it == 0) t0 = t;
            else if (t - t0 > kWaitNs) return false;
        }
    }
}

// Every lane waits (each one acquires the phase); the outcome is made uniform so that a warp never splits around
// warp-collective instructions.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity)
{
    return __all_sync(0xffffffffu, mbar_wait(bar, parity));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// TMA gather of four rows (box: one row of the tensor map's box width) into consecutive shared rows.  The shared
// destination must be 128-byte aligned and the rows inside the tensor [0, rows): a request that breaks either is
// counted in *bad and not issued (its bytes never arrive, so the waiting role times out and the batch fails).
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap *map, int col, int r0, int r1, int r2, int r3,
                                            uint64_t *bar, int rows, unsigned long long *bad)
{
    if ((dst & 127u) != 0u || (unsigned)r0 >= (unsigned)rows || (unsigned)r1 >= (unsigned)rows ||
        (unsigned)r2 >= (unsigned)rows || (unsigned)r3 >= (unsigned)rows) {
        atomicAdd(bad, 1ull);
        return;
    }
    asm volatile("cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
                 "l"(map), "r"(col), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: start >> 4, leading byte offset 16 (unused for swizzled K-major), stride byte
// offset 1024 (8-row groups of 128-byte rows), version bits 46-48 = 0b001, 128-byte swizzle (mode 2, bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A = B = f16, K-major, N >> 3 (bits 17-22), M >> 4
// (bits 24-28).
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
                 "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

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

__device__ __forceinline__ void raise_abort(Ctl &cl, BatchCounters *ctr)
{
    if (!cl.abort_flag) {
        cl.abort_flag = 1;
        atomicAdd(&ctr->errors, 1ull);
    }
}

// ------------------------------------------------------------------------------------------------ setup role
// One warp prepares group gk into slot gk % 2: lines, thresholds, envelope, run table, A-tile gather.
__device__ void setup_group(Ctl &cl, unsigned char *base, const ImageDev *__restrict__ imgs,
                            const PairDev *__restrict__ pairs, const TmaMaps *__restrict__ maps,
                            const int64_t *__restrict__ item_off, int32_t n_pairs, const int32_t *__restrict__ qorder,
                            int64_t item, int g, unsigned long long &my_exam, unsigned long long *bad)
{
    const int lane = threadIdx.x & 31;
    const int pi = pair_of_item(item_off, n_pairs, item);
    const PairDev &P = pairs[pi];
    const ImageDev &A = imgs[P.a];
    const ImageDev &B = imgs[P.b];
    const int q0 = (int)(item - item_off[pi]) * kM;
    const float d = P.d;
    const float W = (float)B.width, H = (float)B.height;
    float F[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) F[t] = P.F[t];
    if (lane < 9) cl.F[g][lane] = F[lane];

    // rows lane, lane + 32, lane + 64, lane + 96: issue the independent loads first
    int s4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int k = q0 + lane + 32 * t;
        s4[t] = k < P.n_a ? qorder[P.qoff + k] : -1;
    }
    float2 q4[4];
    int n4[4], o4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int s = s4[t];
        q4[t] = s >= 0 ? A.xy[s] : make_float2(0.0f, 0.0f);
        n4[t] = s >= 0 ? A.norm256[s] : 0;
        o4[t] = s >= 0 ? A.perm[s] : -1;
    }
    int votes = 0, nnorm = 0, full = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int r = lane + 32 * t;
        float *L = cl.ln[g][r];
        if (s4[t] >= 0) {
            const BandLine bl = band_line(F, q4[t].x, q4[t].y, d, W, H);
            float lo = bl.thr_lo, hi = bl.thr_hi, la = bl.a, lb = bl.b, lc = bl.c;
            // whole-image rows accept every real keypoint; FP64-only rows send every real keypoint to the FP64
            // decision; both use the zero line (s = 0 for real keypoints, NaN for the sentinel record)
            if (bl.mode == kBandAll) { lo = INFINITY; hi = INFINITY; la = lb = lc = 0.0f; }
            else if (bl.mode == kBandSlow) { lo = -1.0f; hi = INFINITY; la = lb = lc = 0.0f; }
            L[0] = la; L[1] = lb; L[2] = lc; L[3] = lo; L[4] = hi; L[5] = q4[t].x; L[6] = q4[t].y;
            L[7] = bl.mode == kBandNormal ? bl.t_walk : -1.0f;
            if (bl.mode == kBandNormal) { ++nnorm; votes += fabsf(bl.b) >= fabsf(bl.a); }
            else full = 1;
        } else {
            L[0] = L[1] = L[2] = 0.0f; L[3] = L[4] = -1.0f; L[5] = L[6] = 0.0f; L[7] = -2.0f;
        }
        cl.rinfo[g][r][0] = o4[t];
        cl.rinfo[g][r][1] = n4[t];
        cl.aidx[g][r] = s4[t] >= 0 ? s4[t] : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        votes += __shfl_xor_sync(0xffffffffu, votes, o);
        nnorm += __shfl_xor_sync(0xffffffffu, nnorm, o);
        full |= __shfl_xor_sync(0xffffffffu, full, o);
    }
    __syncwarp();
    // chord envelope of the group's strips in the walk frame (u: walked axis, v: the other)
    const int colwise0 = 2 * votes >= nnorm;
    const float ulim0 = colwise0 ? W : H;
    float t0 = -INFINITY, t1 = -INFINITY, b0 = INFINITY, b1 = INFINITY, pad = 0.0f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float *L = cl.ln[g][lane + 32 * t];
        if (!(L[7] >= 0.0f)) continue;
        float pa = colwise0 ? L[0] : L[1], pb = colwise0 ? L[1] : L[0], c = L[2];
        if (pb < 0.0f) { pa = -pa; pb = -pb; c = -c; }
        const float T = L[7];
        if (!(pb > 1e-30f)) { full = 1; continue; }
        const float ib = 1.0f / pb;
        const float e0 = -c * ib, e1 = -fmaf(pa, ulim0, c) * ib, h = T * ib;
        t0 = fmaxf(t0, e0 + h); t1 = fmaxf(t1, e1 + h);
        b0 = fminf(b0, e0 - h); b1 = fminf(b1, e1 - h);
        pad = fmaxf(pad, 8.0f * kU * (fabsf(pa) * ulim0 + fabsf(c) + T) * ib);
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
    const bool fin = isfinite(et0) && isfinite(et1) && isfinite(eb0) && isfinite(eb1);
    const int walk_full = full || (nnorm > 0 && !fin);
    const bool none = nnorm == 0 && !full;
    const int colwise = walk_full ? 1 : colwise0;
    // one run of cells per grid line
    const float cs = (float)(1 << B.cell_shift), inv_cs = 1.0f / cs;
    const int nlines = none ? 0 : walk_full ? 1 : (colwise ? B.gx : B.gy);
    const int ng = colwise ? B.gy : B.gx;
    const float ulim = colwise ? W : H, vlim = colwise ? H : W;
    const int32_t *offs = colwise ? B.col_off : B.row_off;
    int carry = 0;
    for (int base_line = 0; base_line < kMaxRuns; base_line += 32 * 8) {
        int st[8], en[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int kk = base_line + 32 * t + lane;
            st[t] = -1;
            en[t] = 0;
            if (kk < nlines) {
                if (walk_full) {
                    st[t] = -2;
                } else {
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
        }
        // run bounds (independent loads), then start / length
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int s0 = 0, s1 = 0;
            if (st[t] >= 0) { s0 = offs[st[t]]; s1 = offs[en[t]]; }
            else if (st[t] == -2) { s0 = 0; s1 = B.n; }
            st[t] = s0;
            en[t] = s1 - s0;
        }
        // exclusive scan of the lengths, in grid-line order
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int kk = base_line + 32 * t + lane;
            int incl = en[t];
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, s);
                if (lane >= s) incl += u;
            }
            cl.run_start[g][kk] = st[t];
            cl.run_excl[g][kk] = carry + incl - en[t];
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    if (lane == 0) {
        cl.run_excl[g][kMaxRuns] = carry;
        Meta &m = cl.meta[g];
        m.pair = pi;
        m.total = carry;
        m.nchunks = (carry + kN - 1) / kN;
        m.walk_full = walk_full;
        m.colwise = colwise;
        my_exam += (unsigned long long)carry * kM;
    }
    __syncwarp();
    // A tile: 32 quads of rows, two K halves each; lane 0 announces the bytes (and releases the slot data) first
    if (lane == 0) mbar_expect_tx(&cl.grp_full[g], kATx);
    __syncwarp();
    const CUtensorMap *dmap = &maps[P.a].desc;
    const uint32_t abase = smem_u32(base + kOffA + g * 2 * kAHalf);
    const int *ai = cl.aidx[g] + 4 * lane;
#pragma unroll
    for (int h = 0; h < 2; ++h)
        tma_gather4(abase + h * kAHalf + 4 * lane * 128, dmap, 64 * h, ai[0], ai[1], ai[2], ai[3], &cl.grp_full[g], A.n,
                    bad);
}

// ------------------------------------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(kThreads, 1) match_tc_kernel(
    const ImageDev *__restrict__ imgs, const PairDev *__restrict__ pairs, const TmaMaps *__restrict__ maps,
    const int64_t *__restrict__ item_off, int32_t n_pairs, const int32_t *__restrict__ qorder, int64_t item_begin,
    int64_t item_end, int32_t *__restrict__ match_j, BatchCounters *__restrict__ ctr)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    Ctl &cl = *reinterpret_cast<Ctl *>(base + kOffCtl);
    const int4 *rec = reinterpret_cast<const int4 *>(base + kOffRec);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t stride = gridDim.x;
    const int64_t first = item_begin + blockIdx.x;
    const int n_groups = first < item_end ? (int)((item_end - first + stride - 1) / stride) : 0;
    unsigned long long my_cand = 0, my_exam = 0, my_redec = 0;

    if (tid == 0) {
        cl.abort_flag = 0;
        cl.stat[0] = cl.stat[1] = cl.stat[2] = 0ull;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&cl.stage_full[s], 1);
            mbar_init(&cl.stage_empty[s], 1 + kEpiWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&cl.acc_full[b], 1);
            mbar_init(&cl.acc_empty[b], kEpiWarps);
        }
        for (int g = 0; g < kSlots; ++g) {
            mbar_init(&cl.grp_full[g], 1);
            mbar_init(&cl.grp_empty[g], 1 + 1 + kEpiWarps);   // MMA commit, loader, epilogue warps
            mbar_init(&cl.merge_ready[g], kEpiWarps / 2);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&cl.tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = cl.tmem_base;

    if (warp >= kSetupWarp0) {
        // ---------------------------------------------------------------- setup warps: groups gk = j, j + 2, ...
        const int j = warp - kSetupWarp0;
        for (int gk = j; gk < n_groups && !cl.abort_flag; gk += kSlots) {
            const int g = gk % kSlots;
            if (!mbar_wait_warp(&cl.grp_empty[g], ((gk / kSlots) & 1) ^ 1)) { raise_abort(cl, ctr); break; }
            setup_group(cl, base, imgs, pairs, maps, item_off, n_pairs, qorder, first + (int64_t)gk * stride, g,
                        my_exam, &ctr->errors);
        }
    } else if (warp == kLoaderWarp) {
        // ---------------------------------------------------------------- loader warp
        int ck = 0;
        for (int gk = 0; gk < n_groups && !cl.abort_flag; ++gk) {
            const int g = gk % kSlots;
            if (!mbar_wait_warp(&cl.grp_full[g], (gk / kSlots) & 1)) { raise_abort(cl, ctr); break; }
            const Meta m = cl.meta[g];
            const PairDev &P = pairs[m.pair];
            const ImageDev &B = imgs[P.b];
            const CUtensorMap *dmap = &maps[P.b].desc;
            const CUtensorMap *rmap = m.colwise ? &maps[P.b].rec : &maps[P.b].rec_r;
            const int32_t *excl = cl.run_excl[g];
            bool ok = true;
            for (int c = 0; c < m.nchunks; ++c, ++ck) {
                const int s = ck % kStages;
                if (!mbar_wait_warp(&cl.stage_empty[s], ((ck / kStages) & 1) ^ 1)) { ok = false; break; }
                // two consecutive slots per lane: record row (walk layout) and descriptor row (column-major)
                int rrow[2], drow[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int p = c * kN + 2 * lane + e;
                    rrow[e] = B.n;   // sentinel record (NaN coordinates)
                    drow[e] = 0;
                    if (p < m.total) {
                        int pos = p;
                        if (!m.walk_full) {
                            int lo = 0, hi = kMaxRuns;
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (excl[mid] <= p) lo = mid;
                                else hi = mid;
                            }
                            pos = cl.run_start[g][lo] + (p - excl[lo]);
                        }
                        rrow[e] = pos;
                        drow[e] = m.colwise ? pos : B.idx_r[pos];
                    }
                }
                const int r2 = __shfl_down_sync(0xffffffffu, rrow[0], 1), r3 = __shfl_down_sync(0xffffffffu, rrow[1], 1);
                const int d2 = __shfl_down_sync(0xffffffffu, drow[0], 1), d3 = __shfl_down_sync(0xffffffffu, drow[1], 1);
                if (lane == 0) mbar_expect_tx(&cl.stage_full[s], kChunkTx);
                __syncwarp();
                if ((lane & 1) == 0) {
                    const int quad = lane >> 1;   // slots 4 quad .. 4 quad + 3
                    const uint32_t bbase = smem_u32(base + kOffB + s * 2 * kBHalf) + 4 * quad * 128;
                    tma_gather4(bbase, dmap, 0, drow[0], drow[1], d2, d3, &cl.stage_full[s], B.n, &ctr->errors);
                    tma_gather4(bbase + kBHalf, dmap, 64, drow[0], drow[1], d2, d3, &cl.stage_full[s], B.n,
                                &ctr->errors);
                    tma_gather4(smem_u32(base + kOffRec + s * kRecStage + quad * 128), rmap, 0, rrow[0], rrow[1], r2, r3,
                                &cl.stage_full[s], B.n + 1, &ctr->errors);
                }
            }
            if (!ok) { raise_abort(cl, ctr); break; }
            if (lane == 0) mbar_arrive(&cl.grp_empty[g]);   // the loader is done with the run table
        }
    } else if (warp == kMmaWarp) {
        // ---------------------------------------------------------------- MMA warp (one thread issues)
        if (lane == 0) {
            int ck = 0;
            for (int gk = 0; gk < n_groups && !cl.abort_flag; ++gk) {
                const int g = gk % kSlots;
                if (!mbar_wait(&cl.grp_full[g], (gk / kSlots) & 1)) { raise_abort(cl, ctr); break; }
                const int nchunks = cl.meta[g].nchunks;
                const uint32_t abase = smem_u32(base + kOffA + g * 2 * kAHalf);
                bool ok = true;
                for (int c = 0; c < nchunks; ++c, ++ck) {
                    const int s = ck % kStages, b = ck & 1;
                    if (!mbar_wait(&cl.stage_full[s], (ck / kStages) & 1) ||
                        !mbar_wait(&cl.acc_empty[b], ((ck >> 1) & 1) ^ 1)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t bbase = smem_u32(base + kOffB + s * 2 * kBHalf);
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks) {
                        const uint32_t off = (uint32_t)((ks & 3) * 32);
                        mma_f16(tmem + b * kN, smem_desc(abase + (ks >> 2) * kAHalf + off),
                                smem_desc(bbase + (ks >> 2) * kBHalf + off), ks > 0 ? 1u : 0u);
                    }
                    mma_commit(&cl.stage_empty[s]);
                    mma_commit(&cl.acc_full[b]);
                }
                if (!ok) { raise_abort(cl, ctr); break; }
                mma_commit(&cl.grp_empty[g]);   // the A tile is free once this group's MMAs are done
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- epilogue warps
        const int quadrant = warp & 3, h = warp >> 2;
        const int row = 32 * quadrant + lane;
        const uint32_t tmem_lane = tmem + ((uint32_t)(32 * quadrant) << 16) + 32 * h;
        int ck = 0;
        for (int gk = 0; gk < n_groups && !cl.abort_flag; ++gk) {
            const int g = gk % kSlots;
            if (!mbar_wait_warp(&cl.grp_full[g], (gk / kSlots) & 1)) { raise_abort(cl, ctr); break; }
            const Meta m = cl.meta[g];
            const PairDev &P = pairs[m.pair];
            const float la = cl.ln[g][row][0], lb = cl.ln[g][row][1], lc = cl.ln[g][row][2];
            const float llo = cl.ln[g][row][3], lhi = cl.ln[g][row][4], qx = cl.ln[g][row][5], qy = cl.ln[g][row][6];
            const int out_i = cl.rinfo[g][row][0];
            // key = (|a'|^2 + |b'|^2 - 2 dot) * 256 + column with dot taken from the f32 accumulator through
            // bits = float_bits(dot + 1.5 * 2^23) = 0x4B400000 + dot, and 512 * 0x4B400000 = 2^31 (mod 2^32)
            const uint32_t Rc = (uint32_t)cl.rinfo[g][row][1] + 0x80000000u + (uint32_t)(32 * h);
            const float d = P.d;
            int k1 = INT_MAX, k2 = INT_MAX, j1 = 0, cnt = 0;
            bool ok = true;
            for (int c = 0; c < m.nchunks; ++c, ++ck) {
                const int s = ck % kStages, b = ck & 1;
                if (!mbar_wait_warp(&cl.acc_full[b], (ck >> 1) & 1)) { ok = false; break; }
                tc_fence_after();
                uint32_t v[32];
                tmem_ld32(tmem_lane + b * kN, v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&cl.acc_empty[b]);
                if (!mbar_wait_warp(&cl.stage_full[s], (ck / kStages) & 1)) { ok = false; break; }   // records visible
                // record of column t: quad slot t / 4 (128 bytes each), entry t % 4
                const int4 *rs = rec + (s * kRecStage + 1024 * h) / 16;
                const int k1_before = k1;
                if (32 * h < m.total - c * kN) {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        const int4 r = rs[(jj >> 2) * 8 + (jj & 3)];
                        const float x = __int_as_float(r.x), y = __int_as_float(r.y);
                        const float sv = fmaf(la, x, fmaf(lb, y, lc));
                        const float as = fabsf(sv);
                        bool inb = as <= llo;
                        if (!inb && as <= lhi) {
                            inb = band_exact_call(cl.F[g], qx, qy, d, x, y);
                            ++my_redec;
                        }
                        const uint32_t bits = (uint32_t)__float_as_int(__int_as_float(v[jj]) + 12582912.0f);
                        const int key = (int)(Rc + (uint32_t)r.z + (uint32_t)jj - 512u * bits);
                        const int km = inb ? key : INT_MAX;
                        k2 = min(k2, max(k1, km));
                        k1 = min(k1, km);
                        cnt += inb;
                    }
                }
                if (k1 < k1_before) {
                    const int t = (k1 & 255) - 32 * h;
                    j1 = rs[(t >> 2) * 8 + (t & 3)].w;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&cl.stage_empty[s]);
            }
            if (!ok) { raise_abort(cl, ctr); break; }
            // merge the two column halves of every row, then the ratio test
            if (h == 1) {
                int32_t *mg = cl.merge[g][row];
                mg[0] = k1; mg[1] = k2; mg[2] = j1; mg[3] = cnt;
                __syncwarp();
                if (lane == 0) mbar_arrive(&cl.merge_ready[g]);
            } else {
                if (!mbar_wait_warp(&cl.merge_ready[g], (gk / kSlots) & 1)) { raise_abort(cl, ctr); break; }
                const int32_t *mg = cl.merge[g][row];
                const int ok1 = mg[0], ok2 = mg[1], oj1 = mg[2];
                const int nk2 = min(max(k1, ok1), min(k2, ok2));
                if (ok1 < k1) { k1 = ok1; j1 = oj1; }
                k2 = nk2;
                cnt += mg[3];
                if (out_i >= 0) {
                    const int64_t D1 = k1 >> 8, D2 = k2 >> 8;
                    int outj = -1;
                    if (cnt >= 2 && (int64_t)P.q * P.q * D1 < (int64_t)P.p * P.p * D2) outj = imgs[P.b].perm[j1];
                    match_j[P.qoff + out_i] = outj;
                    my_cand += (unsigned long long)cnt;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&cl.grp_empty[g]);
        }
    }

    // ---- counters, tensor memory
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_cand += __shfl_xor_sync(0xffffffffu, my_cand, o);
        my_exam += __shfl_xor_sync(0xffffffffu, my_exam, o);
        my_redec += __shfl_xor_sync(0xffffffffu, my_redec, o);
    }
    if (lane == 0) {
        atomicAdd(&cl.stat[0], my_cand);
        atomicAdd(&cl.stat[1], my_exam);
        atomicAdd(&cl.stat[2], my_redec);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
    }
    if (tid == 0) {
        BatchCounters *cc = ctr + (blockIdx.x % kCounterShards);
        atomicAdd(&cc->candidates, cl.stat[0]);
        atomicAdd(&cc->examined, cl.stat[1]);
        atomicAdd(&cc->redecided, cl.stat[2]);
    }
}

cudaError_t prepare()
{
    static cudaError_t once = [] {
        cudaError_t e = cudaFuncSetAttribute(match_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(match_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        return e;
    }();
    return once;
}

}  // namespace

int match_tc_blocks_per_sm() { return 1; }

int match_tc_max_grid_lines() { return kMaxRuns; }

cudaError_t launch_match_tc(const ImageDev *imgs, const PairDev *pairs, const TmaMaps *maps, const int64_t *item_off,
                            int32_t n_pairs, const int32_t *qorder, int64_t item_begin, int64_t item_end, int32_t grid,
                            int32_t *match_j, BatchCounters *ctr, cudaStream_t st)
{
    const int64_t n = item_end - item_begin;
    if (n <= 0) return cudaSuccess;
    cudaError_t e = prepare();
    if (e != cudaSuccess) return e;
    const int64_t g = std::max<int64_t>(1, grid > 0 ? std::min<int64_t>(grid, n) : n);
    match_tc_kernel<<<(unsigned)g, kThreads, kSmemBytes, st>>>(imgs, pairs, maps, item_off, n_pairs, qorder, item_begin,
                                                             item_end, match_j, ctr);
    return cudaGetLastError();
}

}  // namespace gm
