// gm_stream.cu -- candidate streams of the query groups of the tensor-core path (App. A Step 3, per group).
//
// For a group of 128 consecutive (line-sorted) queries the union of their bands lies between the two chords of
// the strips' upper and lower envelopes over the walked image axis: the maximum of linear functions is convex and
// lies below the chord between its end values, the minimum is concave and lies above its chord.  Walking the grid
// column by column (or row by row for steep lines), one run of cells per grid line covers every keypoint any query
// of the group can accept.
//
// The group's 128 rows are four quadrants of 32 consecutive lines (the rows of one epilogue warp of the tcgen05
// matcher); each quadrant has chord envelopes of its own, built the same way.  Every keypoint of the walked runs is
// tested against the four quadrant envelopes: a keypoint outside all four is in no row's band (it only shared a cell
// with the band) and is dropped; the others are ordered by their 4-bit quadrant mask (masks of neighbouring
// quadrants next to each other), so that most 32-position slices of the stream concern one or two quadrants.  After
// the positions, the stream holds one 4-bit mask per 32-position slice (8 per 32-bit word): the quadrants whose
// envelope holds a keypoint of the slice.  An epilogue warp skips the slices its quadrant is not in.  Only the
// order and the dropped keypoints change: every row still tests every keypoint its envelope holds exactly, and the
// order of a row's candidates never changes its result (the top-2 keys are unique up to equal distances, which the
// strict ratio test rejects).
//
// One warp per group, four groups per block.  Space is reserved with one atomic per warp; a stream that would
// overflow the buffer marks its group (the caller grows the buffer and runs the batch again).  Groups that contain
// a whole-image query (d = inf) or an FP64-only line use the whole image and store no stream.
#include <cstdint>

#include "gm_band.cuh"
#include "gm_internal.h"

namespace gm {
namespace {

constexpr int kWarps = 4;
constexpr int kCounterShards = 64;   // the batch's counters are 64 shards (the host sums them): one per block mod 64
constexpr int kMinBlocks = 6;   // resident blocks per SM that __launch_bounds__ asks the register allocation for (80 registers)
constexpr int kG = kTcQueriesPerItem;   // queries per group
constexpr int kMaxLines = 1024;
constexpr int kBinInts = 48;   // per warp: bin counts [16], bin starts [16], bin cursors [16]
constexpr int kSortCap = 1024; // per warp: walked keypoints that are sorted by quadrant mask (longer walks keep walk order)

// Stream order of the 15 nonzero quadrant masks (by the centre, then the width of the quadrant range they span):
// bin r holds the keypoints whose mask is mask_of_bin(r); bin_of(m) is the bin of mask m (15: dropped).  Both
// tables are 16 nibbles of one 64-bit constant, so that a lookup with a different index in every lane is a shift.
constexpr int kBinOfMask[16] = {15, 0, 2, 1, 10, 3, 5, 4, 14, 6, 11, 7, 13, 8, 12, 9};
constexpr int kMaskOfBin[16] = {1, 3, 2, 5, 7, 6, 9, 11, 13, 15, 4, 10, 14, 12, 8, 0};
constexpr unsigned long long pack_nibbles(const int (&t)[16])
{
    unsigned long long v = 0ull;
    for (int i = 0; i < 16; ++i) v |= (unsigned long long)t[i] << (4 * i);
    return v;
}
constexpr unsigned long long kBinPacked = pack_nibbles(kBinOfMask), kMaskPacked = pack_nibbles(kMaskOfBin);
__device__ __forceinline__ int bin_of(unsigned m) { return (int)((kBinPacked >> (4 * m)) & 15ull); }
__device__ __forceinline__ unsigned mask_of_bin(int r) { return (unsigned)((kMaskPacked >> (4 * r)) & 15ull); }

// The pair that owns work item t (the largest k with item_off[k] <= t), found by the whole warp: each round the 32
// lanes probe 32 evenly spaced offsets of the remaining range, so a batch of n pairs takes about log32(n) rounds of
// dependent loads instead of log2(n).  Every lane returns the same pair.
__device__ __forceinline__ int pair_of_item(const int64_t *__restrict__ item_off, int n_pairs, int64_t t)
{
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = n_pairs;   // item_off[lo] <= t < item_off[hi] (item_off[n_pairs] is past every item)
    while (hi - lo > 1) {
        const int span = hi - lo;
        const int probe = lo + (int)(((int64_t)span * lane) >> 5);   // lane 0 probes lo itself
        const bool le = __ldg(item_off + probe) <= t;
        const unsigned bal = __ballot_sync(0xffffffffu, le);
        const int last = 31 - __clz(bal);   // the last lane whose probe is <= t (lane 0 always is)
        const int nlo = __shfl_sync(0xffffffffu, probe, last);
        const int nhi = last < 31 ? __shfl_sync(0xffffffffu, probe, last + 1) : hi;
        lo = nlo;
        hi = max(nhi, nlo + 1);
    }
    return lo;
}

// The quadrant mask of keypoint (u, v) (walk axis u, cross axis v): bit q set iff the point lies between quadrant
// q's two chords at u (qe0 / qd: chord value at u = 0 and its rise over the walked axis; empty quadrants hold -inf
// tops and +inf bottoms, which hold no point).
__device__ __forceinline__ unsigned quad_mask(float u, float v, float inv_ulim, const float (&top0)[4],
                                              const float (&dtop)[4], const float (&bot0)[4], const float (&dbot)[4])
{
    const float f = u * inv_ulim;
    unsigned m = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (v <= fmaf(dtop[q], f, top0[q]) && v >= fmaf(dbot[q], f, bot0[q])) m |= 1u << q;
    return m;
}

__global__ void __launch_bounds__(kWarps * 32, kMinBlocks) stream_kernel(
    const ImageDev *__restrict__ imgs, const PairDev *__restrict__ pairs, const int64_t *__restrict__ item_off,
    int32_t n_pairs, const int32_t *__restrict__ qorder, int64_t item_begin, int64_t item_end,
    GroupDesc *__restrict__ gdesc, int32_t *__restrict__ grows, int32_t *__restrict__ stream, int64_t capacity,
    unsigned long long *__restrict__ used, BatchCounters *__restrict__ ctr, int32_t max_lines)
{
    // per warp: run starts [max_lines], exclusive run offsets [max_lines + 1], the bin table and the walked keypoints
    // (position | bin << 28, in walk order) (sized for the batch's images, so that small grids leave room for more
    // resident blocks)
    extern __shared__ int32_t runs_smem[];
    int32_t *const run_start_w = runs_smem + (threadIdx.x >> 5) * (2 * max_lines + 1 + kBinInts + kSortCap);
    int32_t *const run_excl_w = run_start_w + max_lines;
    int32_t *const bin_cnt = run_excl_w + max_lines + 1, *const bin_start = bin_cnt + 16, *const bin_cur = bin_cnt + 32;
    int32_t *const ent = bin_cnt + kBinInts;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t item = item_begin + (int64_t)blockIdx.x * kWarps + warp;
    const bool active = item < item_end;
    int total = 0, kept = 0, n_words = 0, full = 0, colwise = 1;
    bool sorted = false;   // the walk fits kSortCap: keypoints filtered and ordered by quadrant mask
    const ImageDev *Bp = nullptr;
    const PairDev *Pp = nullptr;
    const ImageDev *Ap = nullptr;
    float qtop0[4], qdtop[4], qbot0[4], qdbot[4], inv_ulim = 0.0f;
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
        inv_ulim = 1.0f / ulim;
        // chord end values of every quadrant (rows lane + 32 t form quadrant t), then of the whole group
        float qt0[4], qt1[4], qb0[4], qb1[4], pad = 0.0f;
        int qn[4];
#pragma unroll
        for (int t = 0; t < kG / 32; ++t) {
            qt0[t] = qt1[t] = -INFINITY;
            qb0[t] = qb1[t] = INFINITY;
            qn[t] = 0;
            if (L4[t].mode != kBandNormal) continue;
            float pa = colwise ? L4[t].a : L4[t].b, pb = colwise ? L4[t].b : L4[t].a, c = L4[t].c;
            if (pb < 0.0f) { pa = -pa; pb = -pb; c = -c; }
            const float T = L4[t].t_walk;
            if (!(pb > 1e-30f)) { full = 1; continue; }
            const float ib = 1.0f / pb;
            const float e0 = -c * ib, e1 = -fmaf(pa, ulim, c) * ib, h = T * ib;
            qt0[t] = e0 + h; qt1[t] = e1 + h;
            qb0[t] = e0 - h; qb1[t] = e1 - h;
            qn[t] = 1;
            pad = fmaxf(pad, 8.0f * kU * (fabsf(pa) * ulim + fabsf(c) + T) * ib);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int t = 0; t < kG / 32; ++t) {
                qt0[t] = fmaxf(qt0[t], __shfl_xor_sync(0xffffffffu, qt0[t], o));
                qt1[t] = fmaxf(qt1[t], __shfl_xor_sync(0xffffffffu, qt1[t], o));
                qb0[t] = fminf(qb0[t], __shfl_xor_sync(0xffffffffu, qb0[t], o));
                qb1[t] = fminf(qb1[t], __shfl_xor_sync(0xffffffffu, qb1[t], o));
                qn[t] |= __shfl_xor_sync(0xffffffffu, qn[t], o);
            }
            pad = fmaxf(pad, __shfl_xor_sync(0xffffffffu, pad, o));
            full |= __shfl_xor_sync(0xffffffffu, full, o);
        }
        float t0 = -INFINITY, t1 = -INFINITY, b0 = INFINITY, b1 = INFINITY;
#pragma unroll
        for (int t = 0; t < kG / 32; ++t) {
            t0 = fmaxf(t0, qt0[t]); t1 = fmaxf(t1, qt1[t]);
            b0 = fminf(b0, qb0[t]); b1 = fminf(b1, qb1[t]);
        }
        const float wpad = pad + 1e-3f + 4.0f * kU * (fabsf(t0) + fabsf(t1) + fabsf(b0) + fabsf(b1));
        const float et0 = t0 + wpad, et1 = t1 + wpad, eb0 = b0 - wpad, eb1 = b1 - wpad;
        if (nnorm > 0 && !(isfinite(et0) && isfinite(et1) && isfinite(eb0) && isfinite(eb1))) full = 1;
        // quadrant chords for the keypoint test: the walk's margin, each quadrant's own rounding term and 0.01 px
#pragma unroll
        for (int t = 0; t < kG / 32; ++t) {
            if (qn[t]) {
                const float qpad =
                    pad + 1.1e-2f + 4.0f * kU * (fabsf(qt0[t]) + fabsf(qt1[t]) + fabsf(qb0[t]) + fabsf(qb1[t]));
                qtop0[t] = qt0[t] + qpad; qdtop[t] = qt1[t] - qt0[t];
                qbot0[t] = qb0[t] - qpad; qdbot[t] = qb1[t] - qb0[t];
            } else {
                qtop0[t] = -INFINITY; qdtop[t] = 0.0f;
                qbot0[t] = INFINITY; qdbot[t] = 0.0f;
            }
        }
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
            sorted = total <= kSortCap;
            if (sorted) {
                // every walked keypoint's quadrant mask and bin, kept in walk order (position | bin << 28).  The
                // keypoints are taken 32 at a time by the whole warp: every non-empty grid line marks its first
                // position, and a running maximum of the marks gives each position its line.
                const float2 *pxy = colwise ? B.xy : B.xy_r;
                for (int e = lane; e < total; e += 32) ent[e] = -1;
                if (lane < 16) bin_cnt[lane] = 0;
                __syncwarp();
                for (int kk = lane; kk < nlines; kk += 32)
                    if (run_excl_w[kk + 1] > run_excl_w[kk]) ent[run_excl_w[kk]] = kk;
                __syncwarp();
                int line_carry = -1;
                for (int e0 = 0; e0 < total; e0 += 32) {   // every position's index in the walked order
                    const int e = e0 + lane;
                    int line = e < total ? ent[e] : -1;
#pragma unroll
                    for (int sft = 1; sft < 32; sft <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, line, sft);
                        if (lane >= sft) line = max(line, u);
                    }
                    line = max(line, line_carry);
                    line_carry = __shfl_sync(0xffffffffu, line, 31);
                    if (e < total) ent[e] = run_start_w[line] + (e - run_excl_w[line]);
                }
                __syncwarp();
                // masks and bins, eight keypoints per lane in flight at a time
                constexpr int kU8 = 8;
                for (int e0 = 0; e0 < total; e0 += 32 * kU8) {
                    float2 pt[kU8];
                    int idx[kU8];
#pragma unroll
                    for (int u = 0; u < kU8; ++u) {
                        const int e = e0 + 32 * u + lane;
                        idx[u] = e < total ? ent[e] : 0;
                        pt[u] = e < total ? __ldg(pxy + idx[u]) : make_float2(0.0f, 0.0f);
                        if (!colwise && e < total) idx[u] = __ldg(B.idx_r + idx[u]);
                    }
#pragma unroll
                    for (int u = 0; u < kU8; ++u) {
                        const int e = e0 + 32 * u + lane;
                        int bin = 15;
                        if (e < total) {
                            const unsigned m = colwise
                                                   ? quad_mask(pt[u].x, pt[u].y, inv_ulim, qtop0, qdtop, qbot0, qdbot)
                                                   : quad_mask(pt[u].y, pt[u].x, inv_ulim, qtop0, qdtop, qbot0, qdbot);
                            bin = bin_of(m);
                            ent[e] = idx[u] | (bin << 28);
                        }
                        const unsigned grp = __match_any_sync(0xffffffffu, bin);
                        if (bin < 15 && (grp & lanemask_lt()) == 0u) bin_cnt[bin] += __popc(grp);
                        __syncwarp();
                    }
                }
                // bin starts (exclusive scan in bin order) and the kept total
                const int cnt = lane < 15 ? bin_cnt[lane] : 0;
                int incl = cnt;
#pragma unroll
                for (int sft = 1; sft < 32; sft <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, incl, sft);
                    if (lane >= sft) incl += u;
                }
                if (lane < 16) {
                    bin_start[lane] = incl - cnt;
                    bin_cur[lane] = incl - cnt;
                }
                kept = __shfl_sync(0xffffffffu, incl, 31);
            } else {
                kept = total;   // a long walk keeps its order and every keypoint; its slices concern every quadrant
            }
            n_words = ((kept + 31) / 32 + 7) / 8;
            __syncwarp();
        }
    }
    // reserve the warp's space with one atomic (no wait for the block's other warps, whose walks differ in
    // length); every stream starts on a 16-byte boundary (positions and mask words are each rounded up to four
    // entries) so that the matcher can stage it with 16-byte copies
    if (!active) return;
    const int reserve = ((kept + 3) & ~3) + ((n_words + 3) & ~3);
    unsigned long long off = 0ull;
    if (lane == 0 && !full && reserve > 0) off = atomicAdd(used, (unsigned long long)reserve);
    off = __shfl_sync(0xffffffffu, off, 0);
    const bool overflow = !full && off + (unsigned long long)reserve > (unsigned long long)capacity;
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
        r.total = overflow ? 0 : (full ? total : kept);
        r.flags = (full ? 1 : 0) | (overflow ? 2 : 0);
        r.p = P.p;
        r.q = P.q;
        for (int t = 0; t < 9; ++t) r.F[t] = P.F[t];
        r.d = P.d;
        r.W = (float)B.width;
        r.H = (float)B.height;
        r.qoff = P.qoff;
        gdesc[item] = r;
        BatchCounters *const cs = ctr + (blockIdx.x % kCounterShards);
        if (overflow) atomicAdd(&cs->overflow, 1ull);
        else if (!full && kept > kTcStagedPositions) atomicAdd(&cs->unstaged, 1ull);
        if (full) atomicAdd(&cs->examined, (unsigned long long)total * kG);
    }
    if (full || overflow || kept == 0) return;
    const ImageDev &B = *Bp;
    int32_t *dst = stream + off;
    if (sorted) {
        // the kept keypoints in bin order: 32 walked keypoints at a time, each lane's rank among the lanes of its bin
        // (walk order within a bin), one cursor update per bin present
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + lane;
            const int x = e < total ? ent[e] : (15 << 28);
            const int bin = (int)((unsigned)x >> 28);
            const unsigned grp = __match_any_sync(0xffffffffu, bin);
            const int rank = __popc(grp & lanemask_lt());
            if (bin < 15) dst[bin_cur[bin] + rank] = x & 0x0fffffff;
            __syncwarp();
            if (bin < 15 && rank == 0) bin_cur[bin] += __popc(grp);
            __syncwarp();
        }
    } else {
        // walk order, every lane the keypoints of its grid lines
        const int nlines = colwise ? B.gx : B.gy;
        for (int kk = lane; kk < nlines; kk += 32) {
            const int e0 = run_excl_w[kk], len = run_excl_w[kk + 1] - e0, st = run_start_w[kk];
            for (int k = 0; k < len; ++k) dst[e0 + k] = colwise ? st + k : B.idx_r[st + k];
        }
    }
    // the 4-bit quadrant mask of every 32-position slice (the masks of the bins it overlaps), 8 slices per word;
    // the elements the epilogue will test: 32 x 32 per quadrant of every slice
    const int n_slices = (kept + 31) / 32;
    unsigned long long elems = 0;
    uint32_t *words = reinterpret_cast<uint32_t *>(dst + ((kept + 3) & ~3));
    for (int w = lane; w < n_words; w += 32) {
        // the word's eight slices [8 w, 8 w + 8): every bin ORs its mask into the slices its range overlaps
        const int s_end = min(8 * w + 8, n_slices);
        uint32_t word = 0u;
        if (!sorted) {
            for (int sl = 8 * w; sl < s_end; ++sl) word |= 0xfu << (4 * (sl - 8 * w));
        } else {
            for (int bin = 0; bin < 15; ++bin) {
                const int b0 = bin_start[bin], n = bin_cnt[bin];
                if (n == 0) continue;
                const int s0 = max(b0 >> 5, 8 * w), s1 = min((b0 + n - 1) >> 5, s_end - 1);
                for (int sl = s0; sl <= s1; ++sl) word |= mask_of_bin(bin) << (4 * (sl - 8 * w));
            }
        }
        for (int sl = 8 * w; sl < s_end; ++sl)
            elems += (unsigned long long)__popc((word >> (4 * (sl - 8 * w))) & 0xfu) * 32ull * 32ull;
        words[w] = word;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) elems += __shfl_xor_sync(0xffffffffu, elems, o);
    if (lane == 0) atomicAdd(&ctr[blockIdx.x % kCounterShards].examined, elems);
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
                                                         (int)(sizeof(int32_t) * kWarps *
                                                               (2 * kMaxLines + 1 + kBinInts + kSortCap)));
    if (attr != cudaSuccess) return attr;
    const size_t smem = sizeof(int32_t) * kWarps * (2 * (size_t)max_lines + 1 + kBinInts + kSortCap);
    stream_kernel<<<(unsigned)((n + kWarps - 1) / kWarps), kWarps * 32, smem, st>>>(
        imgs, pairs, item_off, n_pairs, qorder, item_begin, item_end, gdesc, grows, stream, capacity, used, ctr,
        max_lines);
    return cudaGetLastError();
}

}  // namespace gm
