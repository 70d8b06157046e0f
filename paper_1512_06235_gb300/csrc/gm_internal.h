// gm_internal.h -- device data layout shared by the CUDA kernels and the host orchestration of libgeomatch.
//
// Resident image (App. A Step 1, binned once per image and kept in HBM across every pair that uses it):
//   grid of square cells of 2^cell_shift px; gx = ceil(W / cs) columns, gy = ceil(H / cs) rows;
//   "column-major" order sorts keypoints by (cx, cy, original index): the cells of one grid column are
//   contiguous, so a band walked column by column reads one contiguous run per column;
//   "row-major" order sorts by (cy, cx, original index) for bands walked row by row (steep lines); it holds
//   only coordinates and the column-major position, the descriptors exist once, in column-major order.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace gm {

constexpr int kDim = 128;           // SIFT descriptor length (bytes)
constexpr int kMaxCellShift = 7;    // 128 px cells
constexpr int kMinCellShift = 2;    // 4 px cells
constexpr int kQueriesPerItem = 8;  // queries per work item (SIMT path: one warp each)

struct ImageDev {
    int32_t n, width, height;
    int32_t cell_shift;             // cell size = 1 << cell_shift px
    int32_t gx, gy;
    const float2 *xy;               // [n] column-major order
    const int32_t *perm;            // [n] column-major position -> original index
    const int32_t *inv_perm;        // [n] original index -> column-major position
    const int8_t *desc;             // [n][128] column-major order, recentred b - 128 (bit pattern b ^ 0x80)
    const int32_t *norm;            // [n] sum_k (b_k - 128)^2
    const int32_t *norm256;         // [n] norm * 256 (the tensor-core epilogue's key term)
    const int32_t *col_off;         // [gx*gy + 2]; cell (cx, cy) -> cx*gy + cy (then out-of-image cell, total)
    const float2 *xy_r;             // [n] row-major order
    const int32_t *idx_r;           // [n] row-major position -> column-major position
    const int32_t *row_off;         // [gx*gy + 2]; cell (cx, cy) -> cy*gx + cx
    const uint16_t *desc_h;         // [n][128] fp16 bits of (b - 128), column-major order (tensor-core path)
    const int4 *rec;                // [n + 1] (x, y, norm * 256, position) column-major; [n] = NaN sentinel
    // [n][16] fp16, column-major: (-(norm >> 11), -(norm & 2047) / 2, 1024, 0 ...), so that the dot product with the
    // row (1024, 1, 4096, 0 ...) is 2^22 - norm / 2 exactly (the whole-image matcher's extra K step)
    const uint16_t *ext_h;
};

// TMA descriptors of one resident image (tcgen05 path): 64-row boxes of the fp16 descriptor rows (64 elements
// wide, 128-byte swizzle) and of the records (read as FP32 so that rows past the end come back as NaN).
// CUtensorMap carries the alignment TMA requires.
struct TmaMaps {
    CUtensorMap desc_tile;   // fp16 descriptors, 64 x 64 box (contiguous chunks)
    CUtensorMap desc_row;    // fp16 descriptors, 64 x 1 box (gather4 of scattered rows)
    CUtensorMap rec_tile;    // records, 4 x 64 box, NaN past the end
    CUtensorMap ext_tile;    // the fp16 norm rows (ext_h), 16 x 64 box, 32-byte swizzle, zeros past the end
};

struct PairDev {
    int32_t a, b;                   // slots in the device image table
    float F[9];
    float d;                        // band half-width in px, >= 0 or +inf
    int32_t p, q;                   // ratio p/q, 0 <= p < q
    int64_t qoff;                   // offset of this pair's queries in the per-query arrays
    int32_t n_a;                    // |A|
    int32_t flags;
};

// Counters accumulated by the kernels of one batch (unsigned long long for atomicAdd).
struct BatchCounters {
    unsigned long long candidates;  // sum_i |C_i|
    unsigned long long examined;    // points visited by the cell walk
    unsigned long long redecided;   // FP64 re-decisions
    unsigned long long errors;      // device-side argument / bound violations (must stay 0)
    unsigned long long overflow;    // groups whose candidate stream did not fit the stream buffer
    unsigned long long unstaged;    // tcgen05 groups whose stream is longer than kTcStagedPositions
};

// Self-contained description of one query group of the tensor-core path (written by the stream kernel, so the
// matching kernel needs no pair or image table lookups): stream[off .. off + total) holds column-major positions
// in image B; flags bit 0: the group uses the whole image (positions 0 .. total-1, nothing stored), bit 1: the
// stream did not fit the buffer (the batch must be run again with a larger buffer).  The group's query rows
// (column-major positions in A, -1 past the end of the pair) are stored separately, kTcQueriesPerItem per group.
struct alignas(16) GroupDesc {
    int64_t off;                    // stream offset
    const int4 *a_rec;              // A's point records (x, y, |a'|^2 * 256, position)
    const int32_t *a_perm;          // A: column-major position -> original index
    const uint16_t *a_desc;         // A's fp16 descriptor rows
    const uint16_t *b_desc;         // B's fp16 descriptor rows
    const int4 *b_rec;              // B's point records
    const int32_t *b_perm;          // B: column-major position -> original index
    int32_t a_slot, b_slot;         // image slots (TMA descriptor table)
    int32_t a_n, b_n;
    int32_t total, flags;
    int32_t p, q;                   // ratio p/q
    float F[9];
    float d, W, H;                  // band half-width, size of image B
    int64_t qoff;                   // the pair's offset in the per-query output
};
constexpr int kTcQueriesPerItem = 128;
// Candidate positions a tcgen05 group stages in shared memory; a longer stream is read from global memory.
constexpr int kTcStagedPositions = 1024;

// ---- launchers (host functions defined in the .cu files) ---------------------------------------------------
// Image registration, many images per launch, in two phases so that invalid input never touches a destination:
// the count phase histograms the cells and counts keypoints outside [0,W) x [0,H) per image; the build phase
// (only after every count was read as 0) scans, scatters and copies the descriptors.  Keypoint g of the batch
// belongs to image k with kp_base[k] <= g < kp_base[k+1]; the image's two count arrays (column-major then
// row-major, m + 1 entries each, m = gx * gy + 1) sit at cnt_base in the shared work array.  All pointers are
// device pointers.
struct BucketJob {
    const float2 *xy_raw;
    const uint8_t *desc_raw;
    int32_t n, width, height, cell_shift, gx, gy, m;
    int32_t pad_;
    int64_t kp_base, cnt_base;
    float2 *xy, *xy_r;
    int32_t *perm, *inv_perm, *norm, *norm256, *col_off, *idx_r, *row_off;
    int8_t *desc;
    uint16_t *desc_h;
    int4 *rec;
    uint16_t *ext_h;
};

// Exclusive scan of m int32 counts into off[0 .. m] (off[m] = total); bsum holds m / 1024 + 1 entries.
cudaError_t launch_exclusive_scan(const int32_t *cnt, int32_t m, int32_t *off, int32_t *bsum, cudaStream_t st);

// Counts of every image of the batch (work[0, S) and bad[0, K) are cleared first); bad[k] counts image k's
// keypoints outside its image.  kp_prefix[K + 1] and cnt_prefix[K + 1] are the jobs' kp_base / cnt_base with the
// totals at [K].
cudaError_t launch_bucket_batch_count(const BucketJob *jobs, const int64_t *kp_prefix, int32_t K, int64_t n_total,
                                      int32_t *work, int64_t S, unsigned long long *bad, cudaStream_t st);
// Offsets, scatters, descriptor copies and records of every image (after launch_bucket_batch_count); scan needs
// S + 1 entries and bsum S / 1024 + 2; rec_prefix[k] = kp_prefix[k] + k (each image's records end with a sentinel).
cudaError_t launch_bucket_batch_build(const BucketJob *jobs, const int64_t *kp_prefix, const int64_t *cnt_prefix,
                                      const int64_t *rec_prefix, int32_t K, int64_t n_total, int32_t *work, int64_t S,
                                      int32_t *scan, int32_t *bsum, cudaStream_t st);

// Query ordering (App. A Step 2 as an order only): per pair, sorts A's queries by the position of their
// epipolar line in B.  qorder[qoff + k] = column-major position in A of the k-th query.
cudaError_t launch_order(const ImageDev *imgs, const PairDev *pairs, int32_t n_pairs, int32_t *qorder,
                         cudaStream_t st);

// SIMT matching path: one warp per query.  match_j[qoff + i] = original B index or -1 for original A index i.
// Work items are groups of kQueriesPerItem sorted queries; pair k owns items [item_off[k], item_off[k+1]).
// grid > 0: persistent launch of `grid` blocks taking items [item_begin, item_end) from the counter *next
// (zeroed by the caller); grid == 0: one block per item.
cudaError_t launch_match_simt(const ImageDev *imgs, const PairDev *pairs, const int64_t *item_off, int32_t n_pairs,
                              const int32_t *qorder, int64_t item_begin, int64_t item_end, int32_t grid,
                              int32_t *next, int32_t *match_j, BatchCounters *ctr, cudaStream_t st);
int match_simt_blocks_per_sm();

// Tensor-core matching path (mma.sync s8): groups of 16*mt sorted queries (mt = 1 or 2) per work item.
cudaError_t launch_match_mma(int mt, const ImageDev *imgs, const PairDev *pairs, const int64_t *item_off,
                             int32_t n_pairs, const int32_t *qorder, int64_t item_begin, int64_t item_end,
                             int32_t grid, int32_t *next, int32_t *match_j, BatchCounters *ctr, cudaStream_t st);
int match_mma_blocks_per_sm(int mt);

// tcgen05 matching path (warp-specialised, TMA gather4 + tcgen05.mma): groups of kTcQueriesPerItem sorted
// queries per work item, one persistent CTA per SM (grid CTAs take items item_begin + b, + grid, ...).
// The group streams come from launch_stream; every image of the batch must have max(gx, gy) <=
// match_tc_max_grid_lines().  cta_time[0..2] (zeroed by the caller) receive the complement of the earliest CTA
// start, the complement of the first CTA finish and the last CTA finish (globaltimer, ns).
// whole_image: every pair of the batch has d = inf (every group uses the whole target image): the specialised
// kernel adds each target's norm through one more K step and keeps the top-2 on the raw accumulator bits.
// pipe (0 .. kTcPipes - 1) selects the banded kernel's pipeline geometry: (candidate chunks in flight, query groups
// in flight, positions staged per group) = (6, 3, 1024), (8, 2, 1024) or (4, 4, 512).
constexpr int kTcPipes = 3;
cudaError_t launch_match_tc(const TmaMaps *maps, const GroupDesc *gdesc, const int32_t *grows, const int32_t *stream,
                            int64_t item_begin, int64_t item_end, int32_t grid, int32_t *match_j, BatchCounters *ctr,
                            unsigned long long *cta_time, bool whole_image, int32_t pipe, cudaStream_t st);
// Candidate streams of the tcgen05 groups [item_begin, item_end) of a batch (grec is indexed by item); *used
// accumulates the stream entries written (zeroed by the caller).
cudaError_t launch_stream(const ImageDev *imgs, const PairDev *pairs, const int64_t *item_off, int32_t n_pairs,
                          const int32_t *qorder, int64_t item_begin, int64_t item_end, GroupDesc *gdesc, int32_t *grows,
                          int32_t *stream, int64_t capacity, unsigned long long *used, BatchCounters *ctr,
                          int32_t max_lines, cudaStream_t st);
int match_tc_blocks_per_sm();
int match_tc_max_grid_lines();

// Output assembly: counts[p] = matches of pair p, pair_off = exclusive scan (pair_off[n_pairs] = total), then
// rows (i, j) sorted by i into matches.
cudaError_t launch_count_matches(const PairDev *pairs, int32_t n_pairs, const int32_t *match_j, int32_t *counts,
                                 int64_t *pair_off, cudaStream_t st);
cudaError_t launch_write_matches(const PairDev *pairs, int32_t n_pairs, const int32_t *match_j,
                                 const int64_t *pair_off, int32_t *matches, cudaStream_t st);

// Candidate sets of one pair for original queries [q_begin, q_begin + q_count): one bitmap per query over B's
// original indices (words 32-bit words each, zeroed by the caller), then CSR with ascending indices.
cudaError_t launch_candidates_bitmap(const ImageDev *imgs, const PairDev *pair, int32_t q_begin, int32_t q_count,
                                     uint32_t *bitmap, int32_t words, BatchCounters *ctr, cudaStream_t st);
cudaError_t launch_bitmap_to_csr_count(const uint32_t *bitmap, int32_t q_count, int32_t words, int32_t *counts,
                                       int64_t *off, cudaStream_t st);
cudaError_t launch_bitmap_to_csr_fill(const uint32_t *bitmap, int32_t q_count, int32_t words, const int64_t *off,
                                      int32_t *cand, cudaStream_t st);

}  // namespace gm
