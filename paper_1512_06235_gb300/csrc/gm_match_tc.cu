// gm_match_tc.cu -- tcgen05 matching path: warp-specialised pipeline of 128-query x 64-candidate tensor-core tiles
// (128-candidate tiles when every pair is matched against the whole target image).
//
// App. A Steps 3-4 for groups of 128 consecutive queries of one pair (queries sorted by the position of their
// epipolar line, so a group's bands nearly coincide; every query keeps its own exact band).  One persistent CTA
// per SM runs four roles that hand work to each other through mbarriers:
//
//   worker warps (3): group set-up and chunk loads, round robin (a TMA or cp.async issue stream of one warp
//       moves only about 6 bytes per cycle, so one warp cannot keep the pipeline fed).  Set-up of a group: its
//       coordinates, norms and output indices, the TMA gather4 of its 128 query descriptors (recentred, fp16:
//       integers in [-128, 127] are exact) into the slot's A tile (128-byte-swizzled K-major layout), and a copy of
//       its candidate stream (positions computed beforehand by gm_stream.cu: the chord-bounded cell walk of the
//       whole group) into shared memory; everything comes from the group's descriptor, loaded well before the slot
//       frees.  Chunk loads: 64 stream positions at a time, the fp16 descriptor rows (two K halves) and a 16-byte
//       record per candidate (x, y, |b'|^2 * 256, position) into a 6-stage ring: scattered rows by TMA gather4
//       (records by cp.async, completion through cp.async.mbarrier.arrive), the contiguous rows of whole-image
//       groups by TMA tile loads (64-row boxes, 128-byte swizzle; rows past the image read as NaN records); slots
//       past the end of a stream get the image's NaN sentinel record;
//   MMA warp (one elected thread): eight tcgen05.mma.kind::f16 per chunk (M = 128, N = 64, K = 16 each; N = 128
//       for whole-image batches, whose chunks would otherwise be bound by the issue of the MMAs), f32
//       accumulation into one of four tensor-memory buffers.  Products are integers of magnitude <= 2^14 and partial
//       sums <= 2^21 < 2^24, so the accumulator holds the exact integer dot product a'.b';
//   epilogue warps (4 lane quadrants x the chunk's 32-column blocks: 8, or 16 for whole-image batches): each thread
//       derives its query's FP32 line and
//       exact-decision thresholds (gm_band.cuh), then per chunk tcgen05.ld of 32 accumulator columns and per element
//       the FP32 band test, D = |a'|^2 + |b'|^2 - 2 a'.b' packed with the column into one int32 key and a masked
//       running top-2 (two interleaved accumulators, no branch in the loop); the rare elements inside the FP32 error
//       margin are re-decided in FP64 afterwards; at the end of the group the two column halves merge and the
//       integer ratio test q^2 D1 < p^2 D2 decides (Sec. 2.3).  With an unbounded band (d = inf: exhaustive
//       matching, the coarse stage) every real keypoint is a candidate and the per-element band test is skipped.
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
constexpr int kAcc = 4;             // accumulator buffers in tensor memory
constexpr int kMaxGridLines = 1024; // grid lines a group walk may cross (gm_stream.cu)
constexpr int kCounterShards = 64;
constexpr unsigned long long kWaitNs = 1000000000ull;   // one second
constexpr int kFilterMinTotal = 4096;   // whole-image targets from this size test each block's maximum first

constexpr int kAHalf = kM * 128;                    // one K half of a query tile (bytes)

// Pipeline geometry of one kernel instantiation: candidate chunks in flight (stages), query groups in flight
// (slots) and the candidate positions a slot stages in shared memory.  The banded kernel comes in the geometries of
// kTcPipes (gm_autotune times them; GM_OPT_TC_PIPE picks one); the whole-image kernel has its own (N = 128).
//
// Shared-memory layout.  Banded batches: the slots' A tiles, the candidate chunks, a 16-byte record per candidate of
// every chunk, then the control block (with each slot's staged candidate positions).  Whole-image batches
// (kWhole): the records give way to each chunk's fp16 norm rows (32 bytes per candidate, 32-byte swizzle) and the
// constant A block of the norm step (kM rows of 32 bytes); no positions are staged.
template <bool W, int STG, int SLT, int POS>
struct TcCfg {
    static constexpr bool kWhole = W;
    // candidates per chunk: 64 for banded batches (the epilogue skips 32-column slices); 128 for whole-image ones,
    // whose MMA thread would otherwise spend most of a chunk's time issuing instructions of N = 64
    static constexpr int kN = W ? 128 : 64;
    static constexpr int kBHalf = kN * 128;                 // one K half of a candidate chunk
    static constexpr int kTmemCols = kAcc * kN;             // 256 or 512 columns of tensor memory
    // warp roles: epilogue warps 0 .. kEpiWarps - 1 (4 lane quadrants x kN / 32 column blocks of 32), then the
    // first worker, the MMA warp and the other two workers.  Whole-image batches: 16 epilogue warps, 20 warps of at
    // most 102 registers; banded: 8, 12 warps of at most 168 registers
    static constexpr int kEpiWarps = 4 * (kN / 32);
    static constexpr int kWorkers = 3;
    static constexpr int kLoaderWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1, kSetupWarp0 = kEpiWarps + 2;
    static constexpr int kThreads = 32 * (kEpiWarps + 1 + kWorkers);
    static constexpr int kMergeParts = kEpiWarps / 4 - 1;   // column blocks that hand their top-2 to block 0
    static constexpr int kStages = STG, kSlots = SLT, kPosCap = POS;
    static constexpr int kOffA = 0;
    static constexpr int kOffB = kOffA + kSlots * 2 * kAHalf;
    static constexpr int kSide = kWhole ? kN * 32 : kN * 16;   // per stage: norm rows, or records
    static constexpr int kOffSide = kOffB + kStages * 2 * kBHalf;
    static constexpr int kOffAExt = kOffSide + kStages * kSide;
    static constexpr int kOffCtl = kOffAExt + (kWhole ? kM * 32 : 0);
    static constexpr int kPos = kWhole ? 4 : kPosCap;
    static constexpr int kMaskWords = kPosCap / 256 < 4 ? 4 : kPosCap / 256;
    static_assert(kPosCap % kN == 0 && kPosCap % 256 == 0, "staged positions: whole chunks and mask words");
    static_assert(kMaskWords % 4 == 0, "mask rows: whole 16-byte copies");
};

template <class C>
struct CtlT {
    GroupDesc desc[C::kSlots];          // the group in each slot
    float2 qxy[C::kSlots][kM];          // query coordinates
    int32_t rinfo[C::kSlots][kM][2];    // original A index (-1: no query), |a'|^2 * 256
    alignas(16) int32_t aidx[C::kSlots][kM];   // A rows to gather
    int32_t merge[C::kSlots][kM][C::kMergeParts][4];
    alignas(16) int32_t pos[C::kSlots][C::kPos];   // the group's candidate positions (staged)
    // their 32-position slices' quadrant masks, 8 per word; a row is at least 16 bytes (the set-up copies the
    // words with one 16-byte cp.async, which needs a 16-byte-aligned destination of that size)
    alignas(16) uint32_t smask[C::kSlots][C::kMaskWords];
    uint64_t stage_full[C::kStages], stage_empty[C::kStages], acc_full[kAcc], acc_empty[kAcc];
    uint64_t grp_full[C::kSlots], grp_empty[C::kSlots], merge_ready[C::kSlots], pos_full[C::kSlots];
    uint32_t tmem_base;
    volatile int32_t abort_flag;
    unsigned long long stat[3];
};
template <class C>
constexpr int smem_bytes() { return C::kOffCtl + (int)sizeof(CtlT<C>) + 1024; }

// the banded geometries (index = GM_OPT_TC_PIPE) and the whole-image one
using TcPipe0 = TcCfg<false, 6, 3, 1024>;
using TcPipe1 = TcCfg<false, 8, 2, 1024>;
using TcPipe2 = TcCfg<false, 4, 4, 512>;
using TcWhole = TcCfg<true, 3, 2, 1024>;   // N = 128 chunks: three stages of 36 KB, two query slots
static_assert(smem_bytes<TcPipe0>() <= 227 * 1024, "shared memory per CTA");
static_assert(smem_bytes<TcPipe1>() <= 227 * 1024, "shared memory per CTA");
static_assert(smem_bytes<TcPipe2>() <= 227 * 1024, "shared memory per CTA");
static_assert(smem_bytes<TcWhole>() <= 227 * 1024, "shared memory per CTA");

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
        // the suspend-time hint lets the thread sleep until the phase completes (or 20 us pass) instead of
        // spinning on issue slots that the epilogue warps need
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity), "r"(20000u)
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
// The same bounded wait without the suspend-time hint, for waits that a whole warp takes (epilogue, workers): their
// phases complete within a chunk's time, and polling picks them up sooner than a suspended thread wakes.
__device__ __forceinline__ bool mbar_wait_spin(uint64_t *bar, uint32_t parity)
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
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity)
{
    return __all_sync(0xffffffffu, mbar_wait_spin(bar, parity));
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

// TMA tile load of the map's box at (col, row) (2D).  The shared destination must be 128-byte aligned (1024 for
// the 128-byte swizzle) and col a multiple of 16 bytes: a request that breaks either is counted in *bad and not
// issued (its bytes never arrive, so the waiting role times out and the batch fails).
__device__ __forceinline__ void tma_tile(uint32_t dst, const CUtensorMap *map, int col, int row, uint64_t *bar,
                                         uint32_t align, unsigned long long *bad)
{
    if ((dst & (align - 1u)) != 0u || (col & 7) != 0 || row < 0) {
        atomicAdd(bad, 1ull);
        return;
    }
    asm volatile("cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                 "[%4];\n" ::"r"(dst),
                 "l"(map), "r"(col), "r"(row), "r"(smem_u32(bar))
                 : "memory");
}

// TMA gather of four rows (the box is one row of the map's box width) into consecutive shared rows.  The shared
// destination must be 128-byte aligned and the rows inside the tensor [0, rows): a request that breaks either is
// counted in *bad and not issued (its bytes never arrive, so the waiting role times out and the batch fails).
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap *map, int col, int4 r, uint64_t *bar,
                                            int rows, unsigned long long *bad)
{
    if ((dst & 127u) != 0u || (col & 7) != 0 || (unsigned)r.x >= (unsigned)rows || (unsigned)r.y >= (unsigned)rows ||
        (unsigned)r.z >= (unsigned)rows || (unsigned)r.w >= (unsigned)rows) {
        atomicAdd(bad, 1ull);
        return;
    }
    asm volatile("cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
                 "l"(map), "r"(col), "r"(r.x), "r"(r.y), "r"(r.z), "r"(r.w), "r"(smem_u32(bar))
                 : "memory");
}

// Adds bytes to the transaction count of the current phase without arriving.
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 16-byte cp.async.  Both addresses must be 16-byte aligned: a request that is not is counted in *bad and not issued
// (the copy's bytes never arrive; the batch then fails with a device error instead of a misaligned access).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, unsigned long long *bad)
{
    if (((dst | (uint32_t)reinterpret_cast<uintptr_t>(src)) & 15u) != 0u) {
        atomicAdd(bad, 1ull);
        return;
    }
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

// The mbarrier receives one arrival once all cp.async operations issued so far by this thread have completed.
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}



// Shared-memory matrix descriptor: start >> 4, leading byte offset 16 (unused for swizzled K-major), stride byte
// offset 1024 (8-row groups of 128-byte rows), version bits 46-48 = 0b001, 128-byte swizzle (mode 2, bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// The same for a K extent of 32 bytes in the 32-byte-swizzled K-major layout: stride byte offset 256 (8-row groups
// of 32-byte rows), swizzle mode 6.
__device__ __forceinline__ uint64_t smem_desc32(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}

// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A = B = f16, K-major, N >> 3 (bits 17-22), M >> 4
// (bits 24-28).
template <int N>
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
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

template <class Ctl>
__device__ __forceinline__ void raise_abort(Ctl &cl, BatchCounters *ctr)
{
    if (!cl.abort_flag) {
        cl.abort_flag = 1;
        atomicAdd(&ctr->errors, 1ull);
    }
}

// A banded group whose candidate stream fits the slot (and starts on a 16-byte boundary, as gm_stream.cu lays
// them out) has its positions staged in shared memory; otherwise the loader reads them from global memory.
template <int kPosCap>
__device__ __forceinline__ bool positions_staged(const GroupDesc &d)
{
    return (d.flags & 3) == 0 && d.total > 0 && d.total <= kPosCap && (d.off & 3) == 0;
}

// ------------------------------------------------------------------------------------------------ setup role
// Query data of one group, loaded into registers before the slot is free (rows lane + 32 t).
struct SetupData {
    GroupDesc d;
    int s4[4];
    int4 r4[4];
    int o4[4];
};

__device__ __forceinline__ void setup_load(SetupData &sd, const GroupDesc *__restrict__ gdesc,
                                           const int32_t *__restrict__ grows, int64_t item)
{
    const int lane = threadIdx.x & 31;
    sd.d = gdesc[item];
#pragma unroll
    for (int t = 0; t < 4; ++t) sd.s4[t] = __ldg(grows + item * kM + lane + 32 * t);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int sq = sd.s4[t];
        sd.r4[t] = sq >= 0 ? __ldg(sd.d.a_rec + sq) : make_int4(0, 0, 0, 0);
        sd.o4[t] = sq >= 0 ? __ldg(sd.d.a_perm + sq) : -1;
    }
}

// Writes the group into slot g (the slot must be free): query data, descriptor and the staged candidate positions
// (cp.async); pos_full completes with the 32 lanes' cp.async arrivals and lane 0's release.
template <int kPosCap, class Ctl>
__device__ __forceinline__ void setup_store(Ctl &cl, const SetupData &sd, int g, const int32_t *__restrict__ stream,
                                            unsigned long long *bad)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int r = lane + 32 * t;
        cl.qxy[g][r] = make_float2(__int_as_float(sd.r4[t].x), __int_as_float(sd.r4[t].y));
        cl.rinfo[g][r][0] = sd.o4[t];
        cl.rinfo[g][r][1] = sd.r4[t].z;
        cl.aidx[g][r] = sd.s4[t] >= 0 ? sd.s4[t] : 0;
    }
    if (lane == 0) cl.desc[g] = sd.d;
    if (positions_staged<kPosCap>(sd.d)) {   // the candidate stream, 16 bytes per copy (the tail of the last copy is unused)
        const int4 *src = reinterpret_cast<const int4 *>(stream + sd.d.off);
        const uint32_t dst = smem_u32(cl.pos[g]);
        const int n16 = (sd.d.total + 3) >> 2;
        for (int k = lane; k < n16; k += 32) cp_async16(dst + 16 * k, src + k, bad);
        // and the slice masks after them (at most four words, in the stream's own 16-byte-rounded reservation)
        if (lane == 0) cp_async16(smem_u32(cl.smask[g]), src + n16, bad);
    }
    cp_async_arrive(&cl.pos_full[g]);
    __syncwarp();
    if (lane == 0) mbar_arrive(&cl.pos_full[g]);
}

// ------------------------------------------------------------------------------------------------ kernel
template <class L>
__global__ void __launch_bounds__(L::kThreads, 1) match_tc_kernel(
    const TmaMaps *__restrict__ maps, const GroupDesc *__restrict__ gdesc, const int32_t *__restrict__ grows,
    const int32_t *__restrict__ stream, int64_t item_begin, int64_t item_end, int32_t *__restrict__ match_j,
    BatchCounters *__restrict__ ctr, unsigned long long *__restrict__ cta_time)
{
    using Ctl = CtlT<L>;
    constexpr bool kWhole = L::kWhole;
    constexpr int kStages = L::kStages, kSlots = L::kSlots, kPosCap = L::kPosCap;
    constexpr int kN = L::kN, kBHalf = L::kBHalf, kTmemCols = L::kTmemCols;
    constexpr int kEpiWarps = L::kEpiWarps, kWorkers = L::kWorkers, kLoaderWarp = L::kLoaderWarp,
                  kMmaWarp = L::kMmaWarp, kSetupWarp0 = L::kSetupWarp0;
    const uint64_t t_start = globaltimer();
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    Ctl &cl = *reinterpret_cast<Ctl *>(base + L::kOffCtl);
    const int4 *rec = reinterpret_cast<const int4 *>(base + L::kOffSide);
    constexpr int kRecStage = L::kSide;
    constexpr int kOffA = L::kOffA, kOffB = L::kOffB, kOffRec = L::kOffSide;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t stride = gridDim.x;
    const int64_t first = item_begin + blockIdx.x;
    const int n_groups = first < item_end ? (int)((item_end - first + stride - 1) / stride) : 0;
    unsigned long long my_cand = 0, my_redec = 0;

    if (tid == 0) {
        cl.abort_flag = 0;
        cl.stat[0] = cl.stat[1] = cl.stat[2] = 0ull;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&cl.stage_full[s], 32 * kWorkers);   // every lane of every worker (+ tile bytes)
            // the MMA commit and the epilogue warps (records read); whole-image epilogues read no stage, so the MMA
            // alone frees it and the loads run ahead of the epilogue by the accumulator buffers
            mbar_init(&cl.stage_empty[s], kWhole ? 1 : 1 + kEpiWarps);
        }
        for (int b = 0; b < kAcc; ++b) {
            mbar_init(&cl.acc_full[b], 1);
            mbar_init(&cl.acc_empty[b], kEpiWarps);
        }
        for (int g = 0; g < kSlots; ++g) {
            mbar_init(&cl.pos_full[g], 33);   // the setup warp's 32 cp.async arrivals + its release
            mbar_init(&cl.grp_full[g], kWorkers);   // each worker's arrival with its share of the A tile's bytes
            mbar_init(&cl.grp_empty[g], 1 + kEpiWarps + kWorkers);   // MMA commit, epilogue warps, workers
            mbar_init(&cl.merge_ready[g], 4 * L::kMergeParts);   // the warps of column blocks 1 ..
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (kWhole && tid < 2 * kM) {
        // the constant A block of the norm step: (1024, 1, 4096, 0 ...) in both 16-byte halves of every 32-byte row
        // (so the 32-byte swizzle, which only exchanges the halves, leaves it unchanged); then visible to the
        // tensor core (async proxy)
        *reinterpret_cast<uint4 *>(base + L::kOffAExt + 16 * tid) = make_uint4(0x3C006400u, 0x00006C00u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
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

    if (warp == kLoaderWarp || warp >= kSetupWarp0) {
        // ---------------------------------------------------------------- worker warps
        // A TMA or cp.async issue stream of one warp moves only about 6 bytes per cycle, so the three workers share
        // every copy: worker wk issues the gather4 operations o = wk (mod 3) of each tile and the records e = wk
        // (mod 3) of each chunk.  The set-up of group gk (query data, descriptor, positions) is worker gk mod 3's.
        // Every worker walks every group and chunk in order and arrives on grp_empty when it is done with a group,
        // so a slot is never refilled before every worker has seen its previous contents.
        const int wk = warp == kLoaderWarp ? 0 : 1 + warp - kSetupWarp0;
        int ck = 0;
        bool ok = true;
        SetupData nxt;
        if (wk < n_groups) setup_load(nxt, gdesc, grows, first + (int64_t)wk * stride);   // in flight early
        for (int gk = 0; gk < n_groups && ok && !cl.abort_flag; ++gk) {
            const int g = gk % kSlots;
            if (gk % kWorkers == wk) {
                if (!mbar_wait_warp(&cl.grp_empty[g], ((gk / kSlots) & 1) ^ 1)) { ok = false; break; }
                setup_store<kPosCap>(cl, nxt, g, stream, &ctr->errors);
                if (gk + kWorkers < n_groups) setup_load(nxt, gdesc, grows, first + (int64_t)(gk + kWorkers) * stride);
            }
            // the group's descriptor, query rows and staged positions are in the slot once pos_full completes
            if (!mbar_wait_warp(&cl.pos_full[g], (gk / kSlots) & 1)) { ok = false; break; }
            const GroupDesc &dg = cl.desc[g];
            // whole-image batches: every group reads the whole image (d = inf for every pair)
            const int total = dg.total, nchunks = (total + kN - 1) / kN, full = kWhole ? 1 : dg.flags & 1,
                      b_n = dg.b_n;
            {   // this worker's share of the A tile: operation o = wk + 3 lane < 64 gathers rows 4 (o & 31) + 0..3 of
                // K half o >> 5; grp_full completes with the three workers' arrivals and all the tile's bytes
                const int nops = (2 * kM / 4 - wk + kWorkers - 1) / kWorkers;
                if (lane == 0) mbar_expect_tx(&cl.grp_full[g], (uint32_t)nops * 512u);
                __syncwarp();
                for (int o = wk + kWorkers * lane; o < 2 * kM / 4; o += 32 * kWorkers) {
                    const int q = o & 31, hh = o >> 5;
                    const int4 r4 = *reinterpret_cast<const int4 *>(cl.aidx[g] + 4 * q);
                    tma_gather4(smem_u32(base + kOffA + g * 2 * kAHalf + hh * kAHalf + q * 512),
                                &maps[dg.a_slot].desc_row, 64 * hh, r4, &cl.grp_full[g], dg.a_n, &ctr->errors);
                }
            }
            const CUtensorMap *dmap = &maps[dg.b_slot].desc_tile;
            const CUtensorMap *rmap = &maps[dg.b_slot].rec_tile;
            const CUtensorMap *gmap = &maps[dg.b_slot].desc_row;
            const int4 *brec = dg.b_rec;
            const bool staged = positions_staged<kPosCap>(dg);
            const int32_t *gs = stream + dg.off;
            const int32_t *ps = cl.pos[g];
            for (int c = 0; c < nchunks; ++c, ++ck) {
                const int sb = ck % kStages;
                if (!mbar_wait_warp(&cl.stage_empty[sb], ((ck / kStages) & 1) ^ 1)) { ok = false; break; }
                const uint32_t bstage = smem_u32(base + kOffB + sb * 2 * kBHalf);
                const uint32_t rstage = smem_u32(base + kOffRec + sb * kRecStage);
                if (full) {
                    // contiguous rows: TMA tile loads by worker 0 (rows past the image come back as NaN records)
                    if (wk == 0 && lane == 0) {
                        mbar_expect_tx(&cl.stage_full[sb], 2u * kBHalf + (uint32_t)kRecStage);
#pragma unroll
                        for (int t = 0; t < kN / 64; ++t) {   // 64-row boxes
                            const int r0 = c * kN + 64 * t;
                            tma_tile(bstage + 8192 * t, dmap, 0, r0, &cl.stage_full[sb], 1024u, &ctr->errors);
                            tma_tile(bstage + kBHalf + 8192 * t, dmap, 64, r0, &cl.stage_full[sb], 1024u,
                                     &ctr->errors);
                            if (kWhole)   // the norm rows (zeros past the image's end)
                                tma_tile(rstage + 2048 * t, &maps[dg.b_slot].ext_tile, 0, r0, &cl.stage_full[sb],
                                         256u, &ctr->errors);
                            else
                                tma_tile(rstage + 1024 * t, rmap, 0, r0, &cl.stage_full[sb], 128u, &ctr->errors);
                        }
                    } else {
                        mbar_arrive(&cl.stage_full[sb]);
                    }
                } else {
                    // scattered rows: gather4 operation o = wk + 3 lane < 32 brings rows 4 (o & 15) + 0..3 of K half
                    // o >> 4; record slot e = wk + 3 lane < 64 by cp.async.  Past the end of the stream: descriptor
                    // row 0 and the NaN sentinel record
                    const int lim = total - c * kN;
                    const int32_t *rows = (staged ? ps : gs) + c * kN;
                    const int nops = (kN / 2 - wk + kWorkers - 1) / kWorkers;
                    if (lane == 0) mbar_expect_tx_only(&cl.stage_full[sb], (uint32_t)nops * 512u);
                    __syncwarp();
                    const int o = wk + kWorkers * lane;
                    if (o < kN / 2) {
                        const int q = o & 15, hh = o >> 4;
                        int4 r4;
                        r4.x = 4 * q < lim ? rows[4 * q] : 0;
                        r4.y = 4 * q + 1 < lim ? rows[4 * q + 1] : 0;
                        r4.z = 4 * q + 2 < lim ? rows[4 * q + 2] : 0;
                        r4.w = 4 * q + 3 < lim ? rows[4 * q + 3] : 0;
                        tma_gather4(bstage + hh * kBHalf + q * 512, gmap, 64 * hh, r4, &cl.stage_full[sb], b_n,
                                    &ctr->errors);
                    }
                    const int e = wk + kWorkers * lane;
                    if (e < kN) cp_async16(rstage + e * 16, brec + (e < lim ? rows[e] : b_n), &ctr->errors);
                    cp_async_arrive(&cl.stage_full[sb]);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&cl.grp_empty[g]);
        }
        if (!ok) raise_abort(cl, ctr);
    } else if (warp == kMmaWarp) {
        // ---------------------------------------------------------------- MMA warp (one thread issues)
        if (lane == 0) {
            int ck = 0;
            for (int gk = 0; gk < n_groups && !cl.abort_flag; ++gk) {
                const int g = gk % kSlots;
                if (!mbar_wait(&cl.grp_full[g], (gk / kSlots) & 1)) { raise_abort(cl, ctr); break; }
                const int nchunks = (cl.desc[g].total + kN - 1) / kN;
                const uint32_t abase = smem_u32(base + kOffA + g * 2 * kAHalf);
                bool ok = true;
                for (int c = 0; c < nchunks; ++c, ++ck) {
                    const int s = ck % kStages, b = ck % kAcc;
                    if (!mbar_wait(&cl.stage_full[s], (ck / kStages) & 1) ||
                        !mbar_wait(&cl.acc_empty[b], ((ck / kAcc) & 1) ^ 1)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t bbase = smem_u32(base + kOffB + s * 2 * kBHalf);
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks) {
                        const uint32_t off = (uint32_t)((ks & 3) * 32);
                        mma_f16<kN>(tmem + b * kN, smem_desc(abase + (ks >> 2) * kAHalf + off),
                                smem_desc(bbase + (ks >> 2) * kBHalf + off), ks > 0 ? 1u : 0u);
                    }
                    if (kWhole)   // + 2^22 - |b'|^2 / 2: the constant A block against the chunk's norm rows
                        mma_f16<kN>(tmem + b * kN, smem_desc32(smem_u32(base + L::kOffAExt)),
                                smem_desc32(smem_u32(base + kOffRec + s * kRecStage)), 1u);
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
        const uint32_t tmem_lane = tmem + ((uint32_t)(32 * quadrant) << 16) + 32 * h;   // its 32-column block
        int ck = 0;
        for (int gk = 0; gk < n_groups && !cl.abort_flag; ++gk) {
            const int g = gk % kSlots;
            if (!mbar_wait_warp(&cl.grp_full[g], (gk / kSlots) & 1) ||
                !mbar_wait_warp(&cl.pos_full[g], (gk / kSlots) & 1)) { raise_abort(cl, ctr); break; }
            const GroupDesc &gd = cl.desc[g];
            const int total = gd.total, nchunks = (total + kN - 1) / kN;
            const float d = gd.d;
            const bool unbounded = isinf(d);   // the whole image is every row's candidate set
            // the quadrant masks of the stream's 32-position slices (banded groups): a slice whose mask lacks this
            // warp's quadrant holds no keypoint inside any of its rows' bands, and is skipped
            const bool sliced = (gd.flags & 1) == 0;
            const int n_slices = (total + 31) >> 5;   // slices past the last one hold no keypoint
            const uint32_t *mwords = positions_staged<kPosCap>(gd) ? cl.smask[g]
                                     : reinterpret_cast<const uint32_t *>(stream + gd.off + ((total + 3) & ~3));
            const int out_i = cl.rinfo[g][row][0];
            const float qx = cl.qxy[g][row].x, qy = cl.qxy[g][row].y;
            float la = 0.0f, lb = 0.0f, lc = 0.0f, llo = -1.0f, lhi = -1.0f;   // no query: never inside
            // the row's FP64 line, computed on its first re-decision in the group (FP64 is slow on this GPU and
            // only a few rows need it)
            BandLine64 l64{0.0, 0.0, 0.0, -1.0};
            bool have64 = false;
            if (out_i >= 0) {
                const BandLine bl = band_line(gd.F, qx, qy, d, gd.W, gd.H);
                la = bl.a; lb = bl.b; lc = bl.c; llo = bl.thr_lo; lhi = bl.thr_hi;
                // whole-image rows accept every real keypoint; FP64-only rows send every real keypoint to the FP64
                // decision; both use the zero line (s = 0 for real keypoints, NaN for the sentinel record)
                if (bl.mode == kBandAll) { llo = INFINITY; lhi = INFINITY; la = lb = lc = 0.0f; }
                else if (bl.mode == kBandSlow) { llo = -1.0f; lhi = INFINITY; la = lb = lc = 0.0f; }
            }
            // key = (|a'|^2 + |b'|^2 - 2 dot) * 256 + column with dot taken from the f32 accumulator through
            // bits = float_bits(dot + 1.5 * 2^23) = 0x4B400000 + dot, and 512 * 0x4B400000 = 2^31 (mod 2^32)
            const uint32_t Rc = (uint32_t)cl.rinfo[g][row][1] + 0x80000000u + (uint32_t)(32 * h);
            // whole-image batches keep the largest accumulator bits instead (see below): start below every value
            int k1 = kWhole ? -1 : INT_MAX, k2 = kWhole ? -1 : INT_MAX, j1 = 0, cnt = 0;
            bool ok = true;
            for (int c = 0; c < nchunks; ++c, ++ck) {
                const int s = ck % kStages, b = ck % kAcc;
                if (!mbar_wait_warp(&cl.acc_full[b], (ck / kAcc) & 1)) { ok = false; break; }
                if (sliced) {
                    const int sl = (kN / 32) * c + h;
                    if (sl >= n_slices || ((mwords[sl >> 3] >> (4 * (sl & 7) + quadrant)) & 1u) == 0u) {
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive(&cl.acc_empty[b]);
                            mbar_arrive(&cl.stage_empty[s]);
                        }
                        continue;
                    }
                }
                tc_fence_after();
                uint32_t v[32];
                tmem_ld32(tmem_lane + b * kN, v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&cl.acc_empty[b]);
                const int k1_before = k1;
                const int nvalid = total - c * kN - 32 * h;   // real columns of this block (may exceed 32)
                if (kWhole) {
                    // the accumulator holds 2^22 + a'.b' - |b'|^2 / 2 = 2^22 + (|a'|^2 - D) / 2, exactly (half-
                    // integers below 2^23) and positive, so its bits order like its values: the two smallest
                    // distances are the two largest bit patterns.  No records are read: the column of a new best
                    // gives its position (whole-image groups read the image's rows in order).
                    // one 32-column block: nv real columns (may exceed 32) starting at chunk column col0
                    auto whole_block = [&](const uint32_t (&vv)[32], int nv, int col0) {
                        const int kb = k1;
                        // large targets: the block's largest value first; when no row of the warp beats its best
                        // with it, the block can only raise the second best (0.5 operations per element instead of
                        // 2.5).  A row's best improves in about 32 / t of its t-th block, so the test pays once a row
                        // has many blocks (small targets, such as the coarse stage's views, skip it)
                        const bool filter = total >= kFilterMinTotal;
                        int bm = -1;
                        if (filter && nv >= 32) {
#pragma unroll
                            for (int jj = 0; jj < 32; jj += 2) bm = __vimax3_s32(bm, (int)vv[jj], (int)vv[jj + 1]);
                        }
                        if (filter && nv >= 32 && !__any_sync(0xffffffffu, bm > k1)) {
                            k2 = max(k2, bm);
                            cnt += 32;
                        } else if (nv >= 32) {
                            // two independent top-2 chains (column pairs 4t, 4t + 1 and 4t + 2, 4t + 3), merged after
                            int b1 = -1, b2 = -1;
#pragma unroll
                            for (int jj = 0; jj < 32; jj += 4) {
                                const int u = (int)vv[jj], w = (int)vv[jj + 1], x = (int)vv[jj + 2],
                                          y = (int)vv[jj + 3];
                                const int lo = min(u, w), hi = max(u, w), lo2 = min(x, y), hi2 = max(x, y);
                                k2 = __vimax3_s32(k2, lo, min(k1, hi));
                                k1 = max(k1, hi);
                                b2 = __vimax3_s32(b2, lo2, min(b1, hi2));
                                b1 = max(b1, hi2);
                            }
                            k2 = __vimax3_s32(k2, b2, min(k1, b1));
                            k1 = max(k1, b1);
                            cnt += 32;
                        } else if (nv > 0) {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj) {
                                if (jj < nv) {
                                    const int x = (int)vv[jj];
                                    k2 = max(k2, min(k1, x));
                                    k1 = max(k1, x);
                                }
                            }
                            cnt += nv;
                        }
                        if (k1 > kb) {   // the column of the new best (the lowest one if several are equal)
                            int col = 0;
                            if (nv >= 32) {
#pragma unroll
                                for (int jj = 31; jj >= 0; --jj) col = (int)vv[jj] == k1 ? jj : col;
                            } else {
#pragma unroll
                                for (int jj = 31; jj >= 0; --jj)
                                    if ((int)vv[jj] == k1 && jj < nv) col = jj;
                            }
                            j1 = c * kN + col0 + col;
                        }
                    };
                    whole_block(v, nvalid, 32 * h);
                    continue;
                }
                if (!mbar_wait_warp(&cl.stage_full[s], (ck / kStages) & 1)) { ok = false; break; }   // records
                const int4 *rs = rec + (s * kRecStage) / 16 + 32 * h;
                if (unbounded && nvalid > 0) {
                    // d = inf: every real keypoint is a candidate (Eq. 2 holds for any line), so only the key and
                    // the masked-free top-2 remain; columns past the image's end are skipped
                    int ka1 = k1, ka2 = k2, kb1 = INT_MAX, kb2 = INT_MAX;
                    const int *rz = reinterpret_cast<const int *>(rs) + 2;   // r.z of record jj at rz[4 * jj]
                    if (nvalid >= 32) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            const uint32_t bits = (uint32_t)__float_as_int(__int_as_float(v[jj]) + 12582912.0f);
                            const int key = (int)(Rc + (uint32_t)rz[4 * jj] + (uint32_t)jj - 512u * bits);
                            if (jj & 1) { kb2 = min(kb2, max(kb1, key)); kb1 = min(kb1, key); }
                            else { ka2 = min(ka2, max(ka1, key)); ka1 = min(ka1, key); }
                        }
                        cnt += 32;
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            if (jj < nvalid) {
                                const uint32_t bits = (uint32_t)__float_as_int(__int_as_float(v[jj]) + 12582912.0f);
                                const int key = (int)(Rc + (uint32_t)rz[4 * jj] + (uint32_t)jj - 512u * bits);
                                if (jj & 1) { kb2 = min(kb2, max(kb1, key)); kb1 = min(kb1, key); }
                                else { ka2 = min(ka2, max(ka1, key)); ka1 = min(ka1, key); }
                            }
                        }
                        cnt += nvalid;
                    }
                    k2 = min(min(ka2, kb2), max(ka1, kb1));
                    k1 = min(ka1, kb1);
                } else if (!unbounded && nvalid > 0) {
                    // two interleaved top-2 accumulators (even / odd columns) shorten the dependency chain; bit jj
                    // of mlo marks an element inside by the FP32 test, of mhi one not outside (mhi & ~mlo: within
                    // the error margin, re-decided in FP64 below)
                    int ka1 = k1, ka2 = k2, kb1 = INT_MAX, kb2 = INT_MAX;
                    uint32_t mlo = 0u, mhi = 0u;
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        const int4 r = rs[jj];
                        const float sv = fmaf(la, __int_as_float(r.x), fmaf(lb, __int_as_float(r.y), lc));
                        const float as = fabsf(sv);
                        const bool inb = as <= llo;
                        if (inb) mlo |= 1u << jj;
                        if (as <= lhi) mhi |= 1u << jj;
                        const uint32_t bits = (uint32_t)__float_as_int(__int_as_float(v[jj]) + 12582912.0f);
                        const int key = (int)(Rc + (uint32_t)r.z + (uint32_t)jj - 512u * bits);
                        if (inb) {
                            if (jj & 1) { kb2 = min(kb2, max(kb1, key)); kb1 = min(kb1, key); }
                            else { ka2 = min(ka2, max(ka1, key)); ka1 = min(ka1, key); }
                        }
                        // keep the records' shared-memory loads in blocks of eight: hoisting all 32 (128 registers)
                        // ahead of the arithmetic spills registers
                        if ((jj & 7) == 7) asm volatile("" ::: "memory");
                    }
                    k2 = min(min(ka2, kb2), max(ka1, kb1));
                    k1 = min(ka1, kb1);
                    cnt += __popc(mlo);
                    uint32_t und = mhi & ~mlo;
                    while (und) {   // rare: FP64 re-decision with the row's FP64 line (operation order as the reference)
                        const int jj = __ffs(und) - 1;
                        und &= und - 1u;
                        const int4 r = rs[jj];
                        ++my_redec;
                        if (!have64) {
                            l64 = band_line64(gd.F, qx, qy, d);
                            have64 = true;
                        }
                        if (!band_test64_call(l64.a, l64.b, l64.c, l64.thr, __int_as_float(r.x), __int_as_float(r.y)))
                            continue;
                        // the dot product of element jj: v cannot be indexed at run time, so select it
                        uint32_t vj = 0u;
#pragma unroll
                        for (int t = 0; t < 32; ++t) vj = t == jj ? v[t] : vj;
                        const uint32_t bits = (uint32_t)__float_as_int(__int_as_float(vj) + 12582912.0f);
                        const int key = (int)(Rc + (uint32_t)r.z + (uint32_t)jj - 512u * bits);
                        k2 = min(k2, max(k1, key));
                        k1 = min(k1, key);
                        ++cnt;
                    }
                }
                if (k1 < k1_before) j1 = rs[(k1 & 255) - 32 * h].w;
                __syncwarp();
                if (lane == 0) mbar_arrive(&cl.stage_empty[s]);
            }
            if (!ok) { raise_abort(cl, ctr); break; }
            // merge the column blocks of every row (block 0 takes the others' top-2 in column order), then the
            // ratio test
            if (h > 0) {
                int32_t *mg = cl.merge[g][row][h - 1];
                mg[0] = k1; mg[1] = k2; mg[2] = j1; mg[3] = cnt;
                __syncwarp();
                if (lane == 0) mbar_arrive(&cl.merge_ready[g]);
            } else {
                if (!mbar_wait_warp(&cl.merge_ready[g], (gk / kSlots) & 1)) { raise_abort(cl, ctr); break; }
#pragma unroll
                for (int part = 0; part < L::kMergeParts; ++part) {
                    const int32_t *mg = cl.merge[g][row][part];
                    const int ok1 = mg[0], ok2 = mg[1], oj1 = mg[2];
                    if (kWhole) {   // largest bits first
                        const int nk2 = max(min(k1, ok1), max(k2, ok2));
                        if (ok1 > k1) { k1 = ok1; j1 = oj1; }
                        k2 = nk2;
                    } else {
                        const int nk2 = min(max(k1, ok1), min(k2, ok2));
                        if (ok1 < k1) { k1 = ok1; j1 = oj1; }
                        k2 = nk2;
                    }
                    cnt += mg[3];
                }
                int64_t D1, D2;
                if (kWhole) {   // D = |a'|^2 + 2^23 - 2 (the accumulator's value)
                    const int64_t na = cl.rinfo[g][row][1] >> 8;
                    D1 = na + 8388608 - (int64_t)(2.0f * __int_as_float(k1));
                    D2 = na + 8388608 - (int64_t)(2.0f * __int_as_float(k2));
                } else {
                    D1 = k1 >> 8;
                    D2 = k2 >> 8;
                }
                if (out_i >= 0) {
                    const int64_t pp = gd.p, qq = gd.q;
                    int outj = -1;
                    if (cnt >= 2 && qq * qq * D1 < pp * pp * D2) outj = __ldg(gd.b_perm + j1);
                    match_j[gd.qoff + out_i] = outj;
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
        my_redec += __shfl_xor_sync(0xffffffffu, my_redec, o);
    }
    if (lane == 0) {
        atomicAdd(&cl.stat[0], my_cand);
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
        atomicAdd(&cc->redecided, cl.stat[2]);
        // load balance of the persistent grid: earliest start and first finish (stored complemented, so that
        // atomicMax over a zeroed word gives the minimum) and last finish
        const uint64_t t_end = globaltimer();
        atomicMax(cta_time + 0, ~(unsigned long long)t_start);
        atomicMax(cta_time + 1, ~(unsigned long long)t_end);
        atomicMax(cta_time + 2, (unsigned long long)t_end);
    }
}

template <class L>
cudaError_t prepare()
{
    static cudaError_t once = [] {
        cudaError_t e = cudaFuncSetAttribute(match_tc_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem_bytes<L>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(match_tc_kernel<L>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        return e;
    }();
    return once;
}

template <class L>
cudaError_t launch_cfg(const TmaMaps *maps, const GroupDesc *gdesc, const int32_t *grows, const int32_t *stream,
                       int64_t item_begin, int64_t item_end, int64_t g, int32_t *match_j, BatchCounters *ctr,
                       unsigned long long *cta_time, cudaStream_t st)
{
    const cudaError_t e = prepare<L>();
    if (e != cudaSuccess) return e;
    match_tc_kernel<L><<<(unsigned)g, L::kThreads, smem_bytes<L>(), st>>>(maps, gdesc, grows, stream, item_begin, item_end,
                                                                     match_j, ctr, cta_time);
    return cudaGetLastError();
}

}  // namespace

int match_tc_blocks_per_sm() { return 1; }

int match_tc_max_grid_lines() { return kMaxGridLines; }

cudaError_t launch_match_tc(const TmaMaps *maps, const GroupDesc *gdesc, const int32_t *grows, const int32_t *stream,
                            int64_t item_begin, int64_t item_end, int32_t grid, int32_t *match_j, BatchCounters *ctr,
                            unsigned long long *cta_time, bool whole_image, int32_t pipe, cudaStream_t st)
{
    const int64_t n = item_end - item_begin;
    if (n <= 0) return cudaSuccess;
    const int64_t g = std::max<int64_t>(1, grid > 0 ? std::min<int64_t>(grid, n) : n);
    if (whole_image)
        return launch_cfg<TcWhole>(maps, gdesc, grows, stream, item_begin, item_end, g, match_j, ctr, cta_time, st);
    if (pipe == 1)
        return launch_cfg<TcPipe1>(maps, gdesc, grows, stream, item_begin, item_end, g, match_j, ctr, cta_time, st);
    if (pipe == 2)
        return launch_cfg<TcPipe2>(maps, gdesc, grows, stream, item_begin, item_end, g, match_j, ctr, cta_time, st);
    return launch_cfg<TcPipe0>(maps, gdesc, grows, stream, item_begin, item_end, g, match_j, ctr, cta_time, st);
}

int match_tc_pipes() { return kTcPipes; }

}  // namespace gm
