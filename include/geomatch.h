/*
 * geomatch.h -- C ABI of the GB300 geometry-aware pairwise feature matcher.
 *
 * The library implements the guided matching of Shah, Deshpande and Narayanan, "Multistage SFM: A Coarse-to-Fine
 * Approach for 3D Reconstruction" (arXiv 1512.06235), Sec. 6.2 with the GPU steps of Appendix A:
 *
 *   for each image pair (A, B) with fundamental matrix F and band half-width d, and for every feature i of A,
 *     l   = F (x_i, y_i, 1)^T                              epipolar line of i in B            (Sec. 6.2)
 *     C_i = { j in B : |a x_j + b y_j + c| <= d sqrt(a^2+b^2) }   candidate set               (Eqs. 2-3)
 *     D   = sum_k (A_ik - B_jk)^2 for j in C_i             exact squared L2 over 128 bytes   (Sec. 6.2.2)
 *     (D1, j1), D2 = nearest and second-nearest over C_i                                      (App. A Step 4)
 *     match (i, j1) iff |C_i| >= 2 and q^2 D1 < p^2 D2     ratio test with r = p/q             (Sec. 2.3)
 *
 * Image B's features are binned into a uniform grid (App. A Step 1); each band is walked cell by cell and every
 * visited point gets an exact membership decision (FP32 with a proven error margin, FP64 for points inside the
 * margin), so C_i is exactly the set of Eq. 2 -- not the approximate set C' of the paper's overlapping grids.
 * Results are bit-identical to a plain FP64 evaluation of the definition above.  The paper's approximate search
 * itself (overlapping grids, centre-most cells, one C' per group of nearly equal lines) is gm_match_pairs_approx.
 *
 * Conventions for every entry point
 *   - Every function returns a gm_status; nothing throws across the ABI.  gm_last_error() gives the message of
 *     the last failing call on the calling thread.
 *   - Input arrays are borrowed for the duration of the call only; the context copies what it keeps.
 *   - Output arrays are owned by the caller.  An output pointer may be host memory or device memory of the
 *     context's device; the library detects which.
 *   - Keypoint and match indices are the caller's original per-image indices (0-based).
 *   - One context is bound to one CUDA device and one CUDA stream; calls on one context must not overlap
 *     (except gm_submit / gm_poll, which are thread-safe).
 */
#ifndef GEOMATCH_H
#define GEOMATCH_H

#include <stdint.h>

#if defined(__GNUC__)
#define GM_API __attribute__((visibility("default")))
#else
#define GM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gm_ctx gm_ctx;   /* opaque; owns device state (resident images, workspace, streams) */

typedef enum {
    GM_OK = 0,
    GM_ERR_INVALID = -1,    /* a malformed argument (null pointer, out-of-image keypoint, bad ratio, ...) */
    GM_ERR_NOMEM = -2,      /* an allocation failed, or a caller-provided output is too small */
    GM_ERR_BUDGET = -3,     /* the request does not fit the configured device-memory budget */
    GM_ERR_NOT_FOUND = -4,  /* unknown image id or ticket */
    GM_ERR_CUDA = -5,       /* a CUDA runtime error; the message names the call */
    GM_ERR_TIMEOUT = -6,    /* a bounded wait ran out (host poll or a device-side spin) */
    GM_ERR_CANCELLED = -7,  /* the request was cancelled, or the context shut down before it ran */
    GM_ERR_BUSY = -8        /* the serving queue is full */
} gm_status;

/* Distance paths (option GM_OPT_PATH).  All give identical results. */
enum {
    GM_PATH_AUTO = 0,       /* the fastest path for the batch (currently GM_PATH_TC) */
    GM_PATH_TC = 1,         /* tcgen05.mma kind::f16 tiles, integer-valued operands, f32 accumulation (exact) */
    GM_PATH_MMA = 2,        /* mma.sync m16n8k32 s8 x s8 -> s32 query groups */
    GM_PATH_SIMT = 3        /* one warp per query, dp4a on recentred int8 descriptors */
};

/* Options for gm_set_option. */
enum {
    GM_OPT_PATH = 1,        /* GM_PATH_* */
    GM_OPT_SCHEDULE = 2,    /* 0 = whole batch per launch (default), 1 = one pair per launch (plain form) */
    GM_OPT_CELL_PX = 3,     /* grid cell size of images put afterwards: 4, 8, 16, 32, 64 or 128 px, or 0 =
                               automatic (the default: 4 px, coarser only for images wider than 4096 px) */
    GM_OPT_GRAPH = 4,       /* 1 = replay batches through a captured CUDA graph when the shape repeats */
    GM_OPT_MMA_GROUP = 5,   /* queries per group of the mma path: 16 (default) or 32 */
    GM_OPT_STREAM_CAP = 6,  /* entries of the tcgen05 path's candidate-stream buffer (grown automatically) */
    GM_OPT_EVICT_LRU = 7,   /* 1 = an image put that would exceed the memory budget first evicts the least recently
                               used images (last put or matched), with their coarse views, as gm_image_evict would
                               -- never one of the images being put nor one that an unfinished serving request
                               names; 0 (default) = refuse with GM_ERR_BUDGET */
    GM_OPT_TC_PIPE = 8      /* pipeline geometry of the tcgen05 path: 0 (default) = 6 candidate chunks and 3 query
                               groups in flight, 1024 positions staged per group; 1 = 8 chunks, 2 groups, 1024;
                               2 = 4 chunks, 4 groups, 512 (longer candidate streams are read from global memory) */
};

typedef struct {
    int32_t device;              /* CUDA device ordinal */
    uint64_t mem_budget_bytes;   /* device bytes the context may hold (images + workspace); 0 = no limit */
    int32_t max_inflight;        /* serving: batches that may be on the device at once (>= 1; 0 = 2) */
    void *cuda_stream;           /* cudaStream_t for synchronous calls, or NULL for the context's own stream */
    int32_t path;                /* GM_PATH_* */
    int32_t cell_px;             /* grid cell size in px (power of two, 4..128); 0 = automatic */
    const char *tuner_cache;     /* gm_autotune's settings file (text, appended), or NULL */
} gm_config;

typedef struct {
    int32_t img_a;               /* query image id */
    int32_t img_b;               /* target image id */
    float F[9];                  /* row-major; the epipolar line of (x_A, y_A) in B is F (x_A, y_A, 1)^T */
    float band_px;               /* d >= 0: max point-to-line distance in px (half the band width);
                                    +INFINITY = the whole image (exhaustive matching) */
    uint16_t ratio_num;          /* p; the ratio test accepts iff dist1 / dist2 < p / q */
    uint16_t ratio_den;          /* q; requires 0 <= p < q */
} gm_pair;

typedef struct {
    int64_t n_pairs;             /* pairs in the last gm_match_pairs call */
    int64_t n_queries;           /* sum of |A| over those pairs */
    int64_t n_candidates;        /* sum_i |C_i|: exact candidate comparisons (Eq. 2 set sizes) */
    int64_t n_examined;          /* points visited by the cell walk (a superset of the candidates) */
    int64_t n_redecided;         /* points whose band decision was re-taken in FP64 */
    int64_t n_matches;           /* matches written */
    float ms_device;             /* device time of the whole call (CUDA events on the context stream) */
    float ms_match;              /* device time of the band-walk / distance / top-2 kernel(s) */
    int32_t path_used;           /* GM_PATH_* of the distance kernel that ran */
    int32_t kernel_launches;     /* kernels launched by the call */
    int64_t n_device_errors;     /* device-side bounded waits that ran out (the call then fails with TIMEOUT) */
    int64_t n_stream_reruns;     /* times the batch ran again because its candidate streams overflowed the buffer
                                    (the buffer then grows to what the batch needed) */
    int64_t n_unstaged_groups;   /* tcgen05-path query groups whose candidate stream was too long to stage in shared
                                    memory (their positions are read from global memory) */
    float cta_finish_spread;     /* load balance of the persistent tcgen05 grid: (last CTA finish - first CTA
                                    finish) / (last CTA finish - earliest CTA start); 0 on other paths */
    int32_t reserved0;
} gm_stats;

/* Result of gm_autotune. */
typedef struct {
    int32_t path;                /* GM_PATH_* chosen */
    int32_t mma_group;           /* queries per group of the mma path: 16 or 32 */
    int32_t cell_px;             /* grid cell size chosen: 4, 8 or 16 px */
    float ms;                    /* device time of the batch with these settings (best of the timed runs) */
    int32_t from_cache;          /* 1 if the settings came from the tuner_cache file without timing */
    int32_t tc_pipe;             /* GM_OPT_TC_PIPE chosen (the tcgen05 path's pipeline geometry; 0 on other paths) */
} gm_tune_result;

/* Creates a context on cfg->device.  *out receives the handle.  Errors: GM_ERR_INVALID (null pointer, bad
 * option value), GM_ERR_CUDA (device unavailable). */
GM_API gm_status gm_create(const gm_config *cfg, gm_ctx **out);

/* Frees every device and host resource of the context; pending serving requests end with GM_ERR_CANCELLED. */
GM_API gm_status gm_destroy(gm_ctx *ctx);

/* Sets a tuning option (GM_OPT_*).  GM_ERR_INVALID for an unknown key or value. */
GM_API gm_status gm_set_option(gm_ctx *ctx, int32_t key, int64_t value);

/* Registers image `image_id` (>= 0) and makes it resident on the device (App. A Step 1: the keypoints are binned
 * into grid cells once per image, sorted by cell, and the descriptors are stored in cell order, recentred to int8
 * b - 128, with their squared norms).  Replaces an image already registered under that id.
 *   xy:    float32 [n][2] keypoint coordinates (x, y) in px; every keypoint must satisfy 0 <= x < width and
 *          0 <= y < height (otherwise GM_ERR_INVALID);
 *   scale: float32 [n] keypoint scales (stored, not used by the matching; may be NULL);
 *   desc:  uint8 [n][128] SIFT descriptors, row-major;
 *   on_device: 0 = the three pointers are host memory, 1 = device memory of the context's device (then xy must
 *          be 8-byte and desc 16-byte aligned, otherwise GM_ERR_INVALID).  Page-locked host inputs with those
 *          alignments are read in place by the kernels; other host inputs are staged.
 * n may be 0.  Errors: GM_ERR_INVALID, GM_ERR_BUDGET (the resident image would exceed the budget),
 * GM_ERR_NOMEM, GM_ERR_CUDA. */
GM_API gm_status gm_image_put(gm_ctx *ctx, int32_t image_id, int32_t width, int32_t height, int32_t n,
                       const float *xy, const float *scale, const uint8_t *desc, int32_t on_device);

/* One image of gm_images_put: the arguments of gm_image_put. */
typedef struct {
    int32_t image_id;
    int32_t width, height;
    int32_t n;
    const float *xy;             /* float32 [n][2] */
    const float *scale;          /* float32 [n] or NULL */
    const uint8_t *desc;         /* uint8 [n][128] */
} gm_image;

/* Registers `count` images at once (App. A Step 1 for each; same arguments, layout and errors as gm_image_put,
 * all pointers host memory (on_device = 0) or all device memory (1)).  Every keypoint of every image is checked
 * before anything registered changes; the device work of all images is enqueued back to back, so a batch of
 * images costs two stream synchronisations instead of two per image.  An id given twice is GM_ERR_INVALID. */
GM_API gm_status gm_images_put(gm_ctx *ctx, int32_t count, const gm_image *images, int32_t on_device);

/* Drops image `image_id` from the context.  GM_ERR_NOT_FOUND if unknown. */
GM_API gm_status gm_image_evict(gm_ctx *ctx, int32_t image_id);

/* Whether image `image_id` is resident: GM_OK with *n = its keypoint count (n may be NULL), or GM_ERR_NOT_FOUND. */
GM_API gm_status gm_image_info(gm_ctx *ctx, int32_t image_id, int32_t *n);

/* Pins (pin = 1) or unpins (pin = 0) a resident image: GM_OPT_EVICT_LRU never evicts a pinned image.  Pins count;
 * gm_image_evict drops an image whatever its pins.  Errors: GM_ERR_NOT_FOUND, GM_ERR_INVALID (unpinning an image
 * that is not pinned). */
GM_API gm_status gm_image_pin(gm_ctx *ctx, int32_t image_id, int32_t pin);

/* The resident-image cache: caller images resident, device bytes of all resident images (coarse views included),
 * device bytes of the context's work buffers (they count toward the budget too) and images evicted by
 * GM_OPT_EVICT_LRU so far.  Any pointer may be NULL. */
GM_API gm_status gm_image_cache_stats(gm_ctx *ctx, int64_t *images, int64_t *bytes, int64_t *work_bytes,
                                      int64_t *evicted);

/* Candidate image pairs from point-camera co-visibility (Sec. 6.1): the pairs that gm_match_pairs then matches.
 * For each query image q the candidates are the images i != q that see more than `threshold` of the points q sees
 * (|Points(C_q) & Points(C_i)| > T); only the `top_k` of them with the most co-visible points are kept (ties: the
 * lower image index first), and the result is the set of unique unordered pairs over all queries.
 *   n_cams:     images 0 .. n_cams-1, at most 49152 (each image's co-visible counts are one row of n_cams uint32 in
 *               shared memory; device memory holds the inputs, their camera -> points transpose, O(n_cams) and, per
 *               image q, the images b > q with more than T co-visible points (8 bytes each; T = -1: every pair));
 *   point_off:  int64 [n_points + 1], nondecreasing from 0; point p is seen by point_cams[point_off[p] ..
 *               point_off[p+1]-1] (distinct cameras in [0, n_cams); GM_ERR_INVALID otherwise);
 *   point_cams: int32 [point_off[n_points]];  both host or both device memory;
 *   pairs:      int32 [cap][3] rows (a, b, count), a < b, sorted by (a, b); host or device;
 *   *n_written: number of rows; if it exceeds cap, nothing is written and the call returns GM_ERR_NOMEM.
 * threshold >= -1 (T = -1 admits every image), top_k >= 0. */
GM_API gm_status gm_select_pairs(gm_ctx *ctx, int32_t n_cams, int64_t n_points, const int64_t *point_off,
                                 const int32_t *point_cams, int32_t threshold, int32_t top_k, int32_t *pairs,
                                 int64_t cap, int64_t *n_written);

/* Track merging (the step after pairwise matching, Sec. 6.2): tracks are the connected components of the matches.
 * Nodes are features numbered 0 .. n_nodes-1 (e.g. image-major: node = first node of the image + feature index);
 * every row of `edges` (int64 [n_edges][2]) is a match between two nodes.  labels (int64 [n_nodes]) receives for
 * every node the smallest node index of its component; *n_tracks the number of components with at least two nodes.
 * edges and labels may each be host or device memory.  Errors: GM_ERR_INVALID (an endpoint outside the nodes),
 * GM_ERR_TIMEOUT (a bounded device loop ran out; not expected). */
GM_API gm_status gm_merge_tracks(gm_ctx *ctx, int64_t n_nodes, int64_t n_edges, const int64_t *edges, int64_t *labels,
                                 int64_t *n_tracks);

/* Track triangulation (Sec. 6.3: every merged track becomes a 3D point by linear least squares).
 * Nodes are numbered image-major over image_ids (int32 [n_images], host memory): node = (features of
 * image_ids[0 .. k-1]) + feature index in image image_ids[k] (the caller's keypoint order); n_nodes must equal the
 * total.  labels (int64 [n_nodes]) are those of
 * gm_merge_tracks: every label is the smallest node of its component (a label above its node or negative is
 * GM_ERR_INVALID).  Every component with at least two nodes is a track; tracks are numbered by increasing root.
 * Observation (x, y) in the image with camera P (3 x 4, row-major, double [12] per image in P[n_images][12])
 * contributes the rows x P3 - P1 and y P3 - P2 of A = [A3 | a4]; the point X solves (A3^T A3) X = -A3^T a4 in
 * FP64 (NaN if the system is singular; the FP64 sums run in a data-dependent order, so the last bits may differ
 * between calls).  Outputs (cap rows each): X double [cap][3], roots int64 [cap] (the track's smallest node),
 * n_views int32 [cap]; *n_tracks = number of tracks.  If it exceeds cap, nothing is written and the call returns
 * GM_ERR_NOMEM.  P, labels and the outputs may each be host or device memory (X, roots and n_views all alike, else GM_ERR_INVALID).
 * Errors: GM_ERR_INVALID, GM_ERR_NOT_FOUND (an image not put), GM_ERR_NOMEM, GM_ERR_CUDA. */
GM_API gm_status gm_triangulate(gm_ctx *ctx, int32_t n_images, const int32_t *image_ids, const double *P,
                                int64_t n_nodes, const int64_t *labels, int64_t cap, double *X, int64_t *roots,
                                int32_t *n_views, int64_t *n_tracks);

/* Per-image track triangulation (Sec. 6.3, the step before merging): the paper forms, for every query image, the
 * tracks of its features from the matches found in all its candidate images, and triangulates them image by image
 * (so a feature pair matched in both directions gives the same point twice; merging removes such duplicates).
 * The track of feature k of query image q is the observation (q, k), then (c, j) for every pair (q, c), in the
 * order of the pair list, in which k matched j.  Every track with at least two observations becomes a point by
 * the linear least squares of gm_triangulate, its sums taken in the track's observation order (deterministic).
 * Images, cameras and node numbering as in gm_triangulate (image_ids host memory; node = features of
 * image_ids[0 .. k-1] + feature index).  The pairs and their matches are those of a gm_match_pairs call:
 *   pair_images: int32 [n_pairs][2] (img_a, img_b) image ids, each in image_ids, host memory; ordered pairs, each
 *                listed once, img_a != img_b (GM_ERR_INVALID otherwise); img_a is the query image;
 *   pair_off:    int64 [n_pairs + 1], pair_off[0] = 0, non-decreasing; host or device;
 *   matches:     int32 [pair_off[n_pairs]][2] rows (i_A, j_B), i strictly increasing within each pair, both
 *                inside their images (GM_ERR_INVALID otherwise); host or device (8-byte aligned).
 * Outputs (cap rows each): X double [cap][3], nodes int64 [cap] (the query node of each track, increasing),
 * n_views int32 [cap]; *n_tracks = number of tracks.  If it exceeds cap, nothing is written and the call returns
 * GM_ERR_NOMEM.  X, nodes and n_views all host or all device memory (GM_ERR_INVALID otherwise).
 * Errors: GM_ERR_INVALID, GM_ERR_NOT_FOUND (an image not put), GM_ERR_NOMEM, GM_ERR_BUDGET, GM_ERR_CUDA. */
GM_API gm_status gm_triangulate_image_tracks(gm_ctx *ctx, int32_t n_images, const int32_t *image_ids,
                                             const double *P, int32_t n_pairs, const int32_t *pair_images,
                                             const int64_t *pair_off, const int32_t *matches, int64_t cap, double *X,
                                             int64_t *nodes, int32_t *n_views, int64_t *n_tracks);

/* Coarse stage (Sec. 4): matching of the high-scale features of image pairs without geometry.  Every image keeps
 * its floor(n * eta_pct / 100) features of the largest scale (equal scales: the lower feature index first); an
 * image with fewer than min_features features keeps all of them.  A pair (A, B) is matched in two preemptive
 * batches with an unbounded band (exhaustive nearest / second-nearest search and the pair's ratio test): first
 * A's floor(n * first_pct / 100) highest-scale features against B's kept features; then, only if the first batch
 * gave more than min_matches matches, the rest of A's kept features against the same targets (an image below
 * min_features is matched with all its features in the first batch and has no second).  Requires scales
 * (gm_image_put with scale != NULL, no NaN).  A NULL options pointer means the paper's values. */
typedef struct {
    int32_t eta_pct;        /* kept features, % of the image by scale, 1..100 (paper: 20) */
    int32_t first_pct;      /* first query batch, % of the image by scale, 1..eta_pct (paper: 10) */
    int32_t min_features;   /* images with fewer features keep them all, >= 0 (paper: 1000) */
    int32_t min_matches;    /* the second batch runs after more than this many first-batch matches, >= 0 (paper: 4) */
} gm_coarse_opts;

/* Builds (or refreshes, after an image was put again or with other options) the coarse views of the images
 * (image_ids: int32 [n_images], host memory): the selections above, registered on the device as internal images
 * (they count toward the memory budget; evicting an image drops its views).  gm_match_coarse builds missing views itself; this call lets them be built ahead.
 * Errors: GM_ERR_INVALID (bad options, an image without scales or with a NaN scale), GM_ERR_NOT_FOUND, those of
 * gm_image_put. */
GM_API gm_status gm_coarse_prepare(gm_ctx *ctx, int32_t n_images, const int32_t *image_ids,
                                   const gm_coarse_opts *opts);

/* The selection of one image as ascending feature indices: q1 (first query batch), q2 (second query batch) and t
 * (targets), cap entries each (host or device, all alike, else GM_ERR_INVALID); counts[3] (host) receives their sizes.  If a size
 * exceeds cap nothing is written and the call returns GM_ERR_NOMEM.  Builds the views if needed. */
GM_API gm_status gm_coarse_selection(gm_ctx *ctx, int32_t image_id, const gm_coarse_opts *opts, int32_t *q1,
                                     int32_t *q2, int32_t *t, int32_t cap, int32_t *counts);

/* Coarse matching of n_pairs pairs (img_a, img_b and the ratio of each gm_pair; F and band_px are ignored):
 *   pair_off: int64 [n_pairs + 1]; pair k's rows are pair_off[k] .. pair_off[k+1]-1: the first batch's matches
 *             sorted by the feature index of A, then the second batch's, sorted the same way;
 *   matches:  int32 [cap][2] rows (feature of A, feature of B) in the images' own indices;
 *   second:   int32 [n_pairs] or NULL: 1 where the second batch ran;
 *   *n_written: number of rows; if it exceeds cap, pair_off is written, matches not, and the call returns
 *             GM_ERR_NOMEM.  pair_off, matches and second may each be host or device memory.
 * Errors: those of gm_coarse_prepare and gm_match_pairs. */
GM_API gm_status gm_match_coarse(gm_ctx *ctx, int32_t n_pairs, const gm_pair *pairs, const gm_coarse_opts *opts,
                                 int64_t *pair_off, int32_t *matches, int64_t cap, int64_t *n_written,
                                 int32_t *second);

/* Counters of one gm_match_pairs_approx call. */
typedef struct {
    int64_t n_groups;       /* dual-line groups over all pairs (each shares one candidate set) */
    int64_t n_candidates;   /* sum over queries of |C'| */
    int64_t n_cells;        /* chord samples, i.e. centre-most cells looked up (sum over groups of K + 1) */
} gm_approx_stats;

/* The paper's approximate geometry-aware matching (Sec. 6.2.1 grid-based search, Sec. 6.2.2 dual-line groups,
 * App. A Steps 1-4), next to the exact gm_match_pairs for its recall / speed trade-off.  For a pair with cell
 * half-size h = band_px * cell_scale (FP32):
 *   - B's keypoints are binned into four grids of 2h x 2h cells offset by (0, 0), (h, 0), (0, h), (h, h);
 *   - every query's epipolar line meets B's border [0, W] x [0, H] in a chord whose ends, as positions t1 <= t2
 *     along the border (counter-clockwise from (0, 0)), key the query; queries sorted by (t1, t2, index) form
 *     groups that start wherever t1 or t2 differs from the group's first query by more than 2 px; a query whose
 *     line misses B is a group of its own with no candidates;
 *   - a group's candidate set C' is every keypoint of B in the centre-most of the four cells around each of the
 *     K + 1 equidistant points (K = ceil(|AB| / h)) of its first query's chord;
 *   - every query of the group takes exact squared distances to C', nearest and second-nearest, and the integer
 *     ratio test q^2 D1 < p^2 D2 with |C'| >= 2.
 * All geometry is FP32, each operation rounded in a fixed order (no fused multiply-add).  Output layout, cap and
 * errors as gm_match_pairs; band_px must be finite and h >= 0.5 px; stats may be NULL. */
GM_API gm_status gm_match_pairs_approx(gm_ctx *ctx, int32_t n_pairs, const gm_pair *pairs, float cell_scale,
                                       int64_t *pair_off, int32_t *matches, int64_t cap, int64_t *n_written,
                                       gm_approx_stats *stats);

/* Self-test of the device-side failure path (the paper has no counterpart).  Every wait in the library's kernels
 * gives up after a time limit, records the failure in device memory and returns; the host reports GM_ERR_TIMEOUT and
 * the context stays usable.  This call runs that pattern alone: one device thread waits for a flag with a bounded
 * spin of limit_us microseconds (1 .. 1000000); with set_flag = 1 the host sets the flag first and the call returns
 * GM_OK, with set_flag = 0 nothing sets it and the call returns GM_ERR_TIMEOUT. */
GM_API gm_status gm_selftest_wait(gm_ctx *ctx, int32_t limit_us, int32_t set_flag);

/* Autotuner (a tuning aid; the paper has no counterpart).  Times gm_match_pairs on this batch for every distance
 * path (tc in each of its three pipeline geometries; mma with 16- and 32-query groups; simt) and grid cell size
 * (4, 8, 16 px), `repeats` timed runs each after one warm-up, and leaves the fastest setting in the context:
 * GM_OPT_PATH, GM_OPT_TC_PIPE, GM_OPT_MMA_GROUP and GM_OPT_CELL_PX, with the batch's images re-binned from their
 * resident copies to the chosen cell size.  Every
 * setting gives identical match lists.  With cfg->tuner_cache set, the choice is appended to that text file under
 * the batch's signature (pair count, query and target totals, band sum, image size) and a later call with the same
 * signature applies it without timing (*out->from_cache = 1).  Errors: GM_ERR_INVALID (null pointer, n_pairs < 1,
 * repeats outside [1, 100]), GM_ERR_NOT_FOUND (an image not put), and those of gm_match_pairs / gm_image_put. */
GM_API gm_status gm_autotune(gm_ctx *ctx, int32_t n_pairs, const gm_pair *pairs, int32_t repeats,
                             gm_tune_result *out);

/* Matches n_pairs pairs in one batch (Sec. 6.2; App. A Steps 2-4 for all pairs at once) and writes, in the pairs'
 * order, the match list of every pair sorted by the query index i:
 *   pair_off: int64 [n_pairs + 1]; the matches of pair k are rows pair_off[k] .. pair_off[k+1]-1;
 *   matches:  int32 [cap][2] rows (i_A, j_B) of original keypoint indices;
 *   *n_written: the total number of matches.  If it exceeds cap, nothing is written to `matches`, pair_off is
 *               still written, and the call returns GM_ERR_NOMEM (call again with cap >= *n_written).
 * Both images of every pair must have been put (GM_ERR_NOT_FOUND otherwise); F must be finite, band_px >= 0 or
 * +INFINITY, and 0 <= ratio_num < ratio_den (GM_ERR_INVALID otherwise).  With n_pairs == 0 only pair_off[0]=0
 * and *n_written=0 are written.  The call returns when the outputs are complete. */
GM_API gm_status gm_match_pairs(gm_ctx *ctx, int32_t n_pairs, const gm_pair *pairs, int64_t *pair_off,
                         int32_t *matches, int64_t cap, int64_t *n_written);

/* Candidate sets C_i of one pair (App. A Step 3 output, exact Eq. 2 sets) for queries i in
 * [query_begin, query_begin + query_count) of image A (original indices):
 *   cand_off: int64 [query_count + 1] offsets into cand;
 *   cand:     int32 [cap] B indices (original), ascending within each query;
 *   *n_written: total candidates.  GM_ERR_NOMEM if it exceeds cap (cand_off still written). */
GM_API gm_status gm_band_candidates(gm_ctx *ctx, const gm_pair *pair, int32_t query_begin, int32_t query_count,
                             int64_t *cand_off, int32_t *cand, int64_t cap, int64_t *n_written);

/* gm_band_candidates without any allocation (the paper has no counterpart: this is an interface for callers that
 * must not allocate, e.g. with device memory fully committed or in latency-critical loops where cudaMalloc,
 * cudaFree or cudaHostAlloc would stall).  Same sets, same layout, same errors as gm_band_candidates, except:
 *   cand_off, cand: DEVICE memory of the context's device, or managed memory (GM_ERR_INVALID otherwise),
 *            caller-owned;
 *   scratch: one fixed 4 MiB device array per device, so query_count * ceil(|B| / 32) * 4 + 4 * query_count + 768
 *            bytes must fit in 4 MiB (GM_ERR_INVALID with the sizes otherwise; split the query range);
 *   set-up: gm_create looks up the array's address, which loads it onto the device (4 MiB per device, held until
 *            the process exits, charged to no context's budget); only if that lookup failed does the first call
 *            here retry it (and may then load the array), so that call should come before any stream capture;
 *            a context created after cudaDeviceReset refreshes the address;
 *   calls that overlap in time on one device (any thread or context) race on the scratch: serialise them.
 * The call returns when the outputs are complete. */
GM_API gm_status gm_band_candidates_static(gm_ctx *ctx, const gm_pair *pair, int32_t query_begin,
                                           int32_t query_count, int64_t *cand_off, int32_t *cand, int64_t cap,
                                           int64_t *n_written);

/* Counters and device timings of the last gm_match_pairs call on this context. */
GM_API gm_status gm_get_stats(const gm_ctx *ctx, gm_stats *out);

/* ---- serving: continuous batching ------------------------------------------------------------------------
 * gm_submit queues one pair-match request and returns at once with a ticket.  A scheduler thread admits queued
 * requests into device batches while the device-memory budget and the in-flight batch slots allow, so requests
 * that arrive while other batches run on the GPU join the next batch and overlap with the running ones.  The
 * result of a request is identical to what gm_match_pairs gives for that pair alone.  Thread-safe. */
GM_API gm_status gm_submit(gm_ctx *ctx, const gm_pair *pair, uint64_t *ticket);

/* Waits up to timeout_ms (0 = do not wait, < 0 = wait without limit) for request `ticket`, then writes its
 * matches (int32 [cap][2] rows (i_A, j_B), sorted by i) and *n.  Returns GM_ERR_TIMEOUT if the request is not
 * done yet (the ticket stays valid), GM_ERR_NOMEM if cap < *n (the ticket stays valid), GM_ERR_NOT_FOUND for an
 * unknown or already collected ticket, or the request's own error (a device-side wait that ran out inside its
 * batch is GM_ERR_CUDA here, so that GM_ERR_TIMEOUT from gm_poll always means "not done yet").  A collected
 * ticket is released.
 * If latency_us is not NULL it receives the request's submit-to-completion time in microseconds. */
GM_API gm_status gm_poll(gm_ctx *ctx, uint64_t ticket, int32_t *matches, int64_t cap, int64_t *n, int32_t timeout_ms,
                  double *latency_us);

typedef struct {
    int64_t submitted;               /* requests accepted by gm_submit */
    int64_t completed;               /* requests finished successfully */
    int64_t failed;                  /* requests finished with an error */
    int64_t batches;                 /* device batches launched */
    int64_t max_batch_pairs;         /* largest batch, in requests */
    int64_t peak_inflight_batches;   /* most batches on the device at the same time */
    int64_t rejected_budget;         /* gm_submit refusals: larger than a batch slot's share of the budget */
    int64_t rejected_busy;           /* gm_submit refusals: queue full */
} gm_serving_stats;

/* Counters of the serving loop (all zero before the first gm_submit). */
GM_API gm_status gm_get_serving_stats(gm_ctx *ctx, gm_serving_stats *out);

/* Blocks until every submitted request has completed (the results stay available to gm_poll). */
GM_API gm_status gm_serving_drain(gm_ctx *ctx);

/* Message of the last failing call made by this thread (never NULL). */
GM_API const char *gm_last_error(const gm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* GEOMATCH_H */
