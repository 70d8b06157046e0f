// gm_ctx.h -- host-side context, workspace and batch engine shared by the C ABI (gm_api.cu) and the serving
// loop (gm_serve.cu).  C++ only; not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <condition_variable>
#include <cstdint>
#include <mutex>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/geomatch.h"
#include "gm_internal.h"

namespace gm {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct HostBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool mapped = false;
};

// One device allocation shared by the images that one registration call created; freed with its last image.
struct Slab {
    void *p = nullptr;
    int32_t refs = 0;
};

struct ImageSlot {
    int32_t id = -1;
    int32_t slot = -1;
    ImageDev dev{};
    TmaMaps maps{};
    void *block = nullptr;          // inside slab
    Slab *slab = nullptr;
    size_t bytes = 0;
    const float *scale = nullptr;   // keypoint scales in the caller's order (inside block)
    bool has_scale = false;
    uint64_t gen = 0;               // registration generation (changes on every put of this id)
    uint64_t last_use = 0;          // tick of its last put or batch (least recently used images are evicted first)
    int32_t pins = 0;               // gm_image_pin count: a pinned image is never evicted
};

// Coarse-stage views of one registered image (Sec. 4): its high-scale feature subsets registered as internal
// images (negative ids, invisible to the caller) -- the first query batch, the second query batch and the
// targets -- with the feature index lists that map a view's features back to the image's.  An image below the
// minimum feature count is its own query and target view (lists empty = identity).
struct CoarseViews {
    uint64_t gen = 0;               // generation of the image the views were built from
    int32_t eta = 0, first = 0, min_features = 0;
    bool all = false;
    int32_t id[3] = {0, 0, 0};      // q1, q2, t: internal ids (the image's own id when `all`; 0 when empty)
    int32_t n[3] = {0, 0, 0};
    DevBuf lists;                   // int32: q1, q2, t lists (ascending feature indices)
    const int32_t *list[3] = {nullptr, nullptr, nullptr};
};

// Everything one batch needs on the device and in pinned host memory.  The synchronous API owns one; every
// serving slot owns its own, so batches on different slots can be in flight at the same time.
// Everything a captured batch depends on besides the contents of its pinned tables and device buffers.
struct GraphKey {
    int64_t P, Q, n_items;
    int32_t path, mt, pipe, pad0;
    int64_t grid, stream_cap;
    size_t tab_bytes;
    const void *d_tab, *d_qorder, *d_matchj, *d_counts, *d_off, *rows, *d_ctr, *d_grec, *d_grows, *d_stream, *d_imgs,
        *d_maps, *h_tab, *h_off;
    cudaStream_t stream;
};

struct Workspace {
    DevBuf d_tab;        // pair table (caller's order), pair table (processing order), work-item offsets
    DevBuf d_qorder;     // int32 [Q] query order per pair
    DevBuf d_matchj;     // int32 [Q] per-query decision (original B index or -1), indexed by original A index
    DevBuf d_counts;     // int32 [P]
    DevBuf d_off;        // int64 [P+1]
    DevBuf d_rows;       // int32 [Q][2] match rows (device destination of the synchronous API)
    DevBuf d_ctr;        // BatchCounters [64]
    DevBuf d_next;       // int32 work-queue counter of the persistent kernel
    DevBuf d_grec;       // GroupDesc [items] (tcgen05 path)
    DevBuf d_grows;      // int32 [items][128] query rows of every group (tcgen05 path)
    DevBuf d_stream;     // int32 [stream_cap] candidate streams of the groups (tcgen05 path)
    int64_t stream_cap = 0, stream_used = 0, overflow = 0;
    HostBuf h_tab;       // pinned staging of d_tab
    HostBuf h_off;       // pinned: offsets [P+1] then counters [64]
    HostBuf h_rows;      // mapped pinned rows (serving destination)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // plan of the batch being run
    std::vector<PairDev> pd;
    std::vector<int32_t> proc;   // processing order of the pairs (grouped by image B)
    std::vector<int32_t> sort_tmp, sort_cnt;   // scratch of the counting sorts that build it
    int64_t Q = 0, nitems = 0;
    int32_t n_pairs = 0;
    int32_t max_lines = 1;       // longest grid line count of the planned batch's target images
    bool whole_image = false;    // every pair of the planned batch has d = inf
    int32_t launches = 0;
    int32_t path_used = 0;
    // CUDA graph of the last batch shape (GM_OPT_GRAPH): captured the second time a shape is seen
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{}, gseen{};
    int32_t glaunches = 0;
};

struct Server;

}  // namespace gm

struct gm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t budget = 0;
    int32_t path = GM_PATH_AUTO;
    int32_t schedule = 0;
    int32_t cell_shift = 0;          // 0: automatic per image
    int32_t graph = 0;
    int32_t evict_lru = 0;           // GM_OPT_EVICT_LRU
    uint64_t use_tick = 0;
    int64_t images_evicted = 0;
    int32_t max_inflight = 2;
    int32_t num_sms = 0;
    int32_t mma_mt = 1;             // m16 tiles per query group of the tensor-core path
    int32_t tc_pipe = 0;            // pipeline geometry of the tcgen05 path (GM_OPT_TC_PIPE)

    std::unordered_map<int32_t, gm::ImageSlot *> images;
    std::vector<gm::ImageSlot *> slots;
    gm::DevBuf d_imgs;              // ImageDev table indexed by slot
    gm::DevBuf d_maps;              // TmaMaps table indexed by slot (tcgen05 path)
    size_t bytes_images = 0;
    size_t bytes_work = 0;          // every DevBuf of the context and of the server slots

    gm::Workspace ws;               // synchronous calls
    gm::DevBuf d_stage, d_work, d_bad, d_bitmap, d_tune, d_btab, d_pairs, d_pairs_out, d_pairs_pool, d_tracks, d_tri,
        d_tri_out;
    gm::Workspace ws2;              // second batch of the coarse stage's preemptive schedule (shares ws's stream)
    gm::DevBuf d_coarse_tab, d_coarse_stage, d_coarse_out;
    gm::DevBuf d_approx;            // gm_match_pairs_approx: every array of one call
    gm::DevBuf d_segs;              // image registration: copy segments of the scales
    gm::DevBuf d_selftest;          // gm_selftest_wait: the flag and the status
    cudaStream_t copy_stream = nullptr;   // image registration: descriptor uploads beside the keypoint check
    cudaEvent_t ev_stage = nullptr, ev_desc = nullptr;
    std::unordered_map<int32_t, gm::CoarseViews> coarse;   // by caller's image id
    uint64_t image_gen = 0;
    int32_t next_internal_id = -1;
    std::string tuner_cache;        // gm_autotune's settings file ("" = none)
    gm_stats stats{};
    std::recursive_mutex mu;        // guards images, slots, budget counters and ws

    gm::Server *server = nullptr;
};

namespace gm {

// NVTX range over one entry point (visible in Nsight timelines; a no-op when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

gm_status fail(gm_status st, const char *fmt, ...);
size_t align_up(size_t v, size_t a);
gm_status ensure_dev(gm_ctx *ctx, DevBuf &b, size_t bytes);
gm_status ensure_host(HostBuf &b, size_t bytes, bool mapped = false);
void free_dev(gm_ctx *ctx, DevBuf &b);
void free_host(HostBuf &b);
gm_status workspace_init(Workspace &ws, cudaStream_t stream);
void workspace_free(gm_ctx *ctx, Workspace &ws);
// Device bytes held by the workspace's buffers (counted in the context's bytes_work).
size_t workspace_bytes(const Workspace &ws);

// Validates one pair and fills its device record (without qoff).  Negative image ids (internal images) are
// accepted only with `internal`.
gm_status prepare_pair(gm_ctx *ctx, const gm_pair &pr, int64_t k, PairDev &pd, bool internal = false);
// Validates the pairs and fills ws.pd / ws.Q / ws.nitems.  Caller holds ctx->mu.
gm_status engine_plan(gm_ctx *ctx, Workspace &ws, int32_t n_pairs, const gm_pair *pairs, bool internal = false);
// Plans, launches and completes one batch on ws (reruns with a larger stream buffer on overflow); afterwards
// ws.h_off holds the offsets [P + 1] and ws.d_rows the rows.  Caller holds ctx->mu.
gm_status run_batch(gm_ctx *ctx, Workspace &ws, int32_t n_pairs, const gm_pair *pairs, bool internal, const char *fn);
// Registers `count` images (App. A Step 1); internal images carry negative ids.
gm_status put_images(gm_ctx *ctx, int32_t count, const gm_image *imgs, int32_t on_device, const char *fn,
                     bool internal = false);
// Drops one registered image (caller holds ctx->mu; serving drained by the caller).
void drop_image(gm_ctx *ctx, int32_t image_id);
// Gives up an image's block: the slab is freed with its last image.
void release_block(ImageSlot *img);
bool is_device_ptr(const void *p);
bool is_device_ptr_on(const void *p, int device);
// gm_band_candidates_static's scratch: looks up (and so loads) the array on `device`, which must be current.
void noalloc_setup(int device);
// Enqueues the whole batch on ws.stream: table upload, order, match, count/scan, row writing into rows_dst
// (device memory or mapped host memory with room for ws.Q rows; nullptr = ws.d_rows), then the D2H copy of the
// offsets and counters into ws.h_off.  Nothing waits.  Caller holds ctx->mu.
gm_status engine_launch(gm_ctx *ctx, Workspace &ws, int32_t *rows_dst);
// After ws.stream has completed: the statistics of the batch.
void engine_stats(gm_ctx *ctx, Workspace &ws, gm_stats &S);

// serving
Server *server_start(gm_ctx *ctx);
void server_stop(Server *srv);
gm_status server_submit(Server *srv, const gm_pair &pair, uint64_t *ticket);
gm_status server_poll(Server *srv, uint64_t ticket, int32_t *matches, int64_t cap, int64_t *n, int32_t timeout_ms,
                      double *latency_us);
// Waits until no serving batch is in flight (caller holds ctx->mu, so none can start meanwhile).
void server_drain(Server *srv);
gm_status server_stats(Server *srv, gm_serving_stats *out);
// Waits until every submitted request has completed (caller must not hold ctx->mu).
void server_wait_idle(Server *srv);
// Image ids referenced by serving requests not yet finished (they are never evicted).
void server_referenced(Server *srv, std::unordered_set<int32_t> &ids);
const char *last_error();

}  // namespace gm
