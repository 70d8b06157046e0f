// gm_serve.cu -- serving loop: the continuous-batching scheduler (gm_sched.h) driving the batch engine.
//
// Every scheduler slot owns a Workspace with its own CUDA stream, so up to max_inflight batches run on the device
// at once.  A batch is planned and enqueued under the context lock (so image put / evict, which take the same lock
// and then synchronise every slot stream, never free an image that a launched batch still reads); its match rows
// are written by the compaction kernel straight into mapped pinned host memory, and completion is detected with
// cudaEventQuery (the scheduler never blocks on the device).
//
// Admission: a request costs |A| queries of device workspace.  The budget left after the resident images and the
// context's other work buffers is split evenly over the slots, recomputed before every round of admissions (images
// put or evicted since change it); a batch takes queued requests in arrival order while their total cost fits one
// slot's share, and a request that could never fit a slot of the budget left at server start is refused with
// GM_ERR_BUDGET at submission.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <unordered_set>
#include <vector>

#include "gm_ctx.h"
#include "gm_sched.h"

namespace gm {


namespace {

constexpr int64_t kBytesPerQuery = 16;       // qorder + decision + row (device / mapped host)
constexpr int64_t kMaxSlotQueries = 1 << 22;
constexpr int kMaxBatchPairs = 4096;
constexpr size_t kMaxPending = 1 << 20;

struct GpuEngine {
    struct SlotState {
        Workspace ws;
        cudaEvent_t done_ev = nullptr;
        bool failed = false;
        std::vector<int> idx;   // batch position of every launched pair
    };
    gm_ctx *ctx;
    std::vector<SlotState> slots;

    int64_t cost(const gm_pair &p, gm_status *err)
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        PairDev pd;
        const gm_status st = prepare_pair(ctx, p, 0, pd);
        if (st != GM_OK) {
            *err = st;
            return -1;
        }
        return std::max<int64_t>(pd.n_a, 1);
    }

    // Queries one batch may take now: the budget minus the resident images and the work buffers other than the
    // serving slots' own, split over the slots (the slots' buffers are what this share pays for).
    int64_t slot_capacity()
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        if (!ctx->budget) return kMaxSlotQueries;
        int64_t own = 0;
        for (auto &S : slots) own += (int64_t)workspace_bytes(S.ws);
        const int64_t left =
            (int64_t)ctx->budget - (int64_t)ctx->bytes_images - ((int64_t)ctx->bytes_work - own);
        return std::min<int64_t>(kMaxSlotQueries,
                                 std::max<int64_t>(left, 0) / (int64_t)slots.size() / kBytesPerQuery);
    }

    gm_status launch(int s, std::vector<SchedRequest *> &batch)
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        SlotState &S = slots[s];
        S.failed = false;
        S.idx.clear();
        cudaSetDevice(ctx->device);
        std::vector<gm_pair> pairs;
        for (size_t k = 0; k < batch.size(); ++k) {
            PairDev pd;
            const gm_status st = prepare_pair(ctx, batch[k]->pair, 0, pd);   // images may have changed since submit
            if (st != GM_OK) {
                batch[k]->status = st;
                continue;
            }
            pairs.push_back(batch[k]->pair);
            S.idx.push_back((int)k);
        }
        if (pairs.empty()) {
            S.failed = true;
            return GM_OK;
        }
        gm_status st = engine_plan(ctx, S.ws, (int32_t)pairs.size(), pairs.data());
        if (st == GM_OK) st = ensure_host(S.ws.h_rows, sizeof(int32_t) * 2 * std::max<int64_t>(S.ws.Q, 1), true);
        if (st == GM_OK) st = engine_launch(ctx, S.ws, static_cast<int32_t *>(S.ws.h_rows.p));
        if (st == GM_OK && cudaEventRecord(S.done_ev, S.ws.stream) != cudaSuccess) st = GM_ERR_CUDA;
        if (st != GM_OK) {
            S.failed = true;
            for (int k : S.idx) batch[k]->status = st;
        }
        return GM_OK;
    }

    bool done(int s)
    {
        SlotState &S = slots[s];
        if (S.failed) return true;
        const cudaError_t e = cudaEventQuery(S.done_ev);
        if (e == cudaErrorNotReady) return false;
        if (e != cudaSuccess) S.failed = true;
        return true;
    }

    void collect(int s, std::vector<SchedRequest *> &batch)
    {
        SlotState &S = slots[s];
        if (!S.failed) {
            // a candidate-stream overflow invalidates the batch: grow the buffer and run it again (rare)
            gm_stats tmp;
            engine_stats(ctx, S.ws, tmp);
            for (int attempt = 0; S.ws.overflow && attempt < 2; ++attempt) {
                std::lock_guard<std::recursive_mutex> lk(ctx->mu);
                S.ws.stream_cap = S.ws.stream_used + S.ws.stream_used / 4 + 1024;
                if (engine_launch(ctx, S.ws, static_cast<int32_t *>(S.ws.h_rows.p)) != GM_OK ||
                    cudaStreamSynchronize(S.ws.stream) != cudaSuccess) {
                    S.failed = true;
                    break;
                }
                engine_stats(ctx, S.ws, tmp);
            }
            if (S.ws.overflow || tmp.n_device_errors) S.failed = true;
        }
        if (S.failed) {
            for (int k : S.idx)
                if (batch[k]->status == GM_OK) batch[k]->status = GM_ERR_CUDA;
            return;
        }
        const int64_t *off = static_cast<const int64_t *>(S.ws.h_off.p);
        const int32_t *rows = static_cast<const int32_t *>(S.ws.h_rows.p);
        for (size_t t = 0; t < S.idx.size(); ++t) {
            SchedRequest *r = batch[S.idx[t]];
            r->rows.assign(rows + 2 * off[t], rows + 2 * off[t + 1]);
            r->status = GM_OK;
        }
    }
};

}  // namespace

struct Server {
    GpuEngine eng;
    Scheduler<GpuEngine> *sched = nullptr;
};

Server *server_start(gm_ctx *ctx)
{
    Server *srv = new Server();
    srv->eng.ctx = ctx;
    const int n = std::max(1, ctx->max_inflight);
    srv->eng.slots.resize(n);
    for (auto &S : srv->eng.slots) {
        if (workspace_init(S.ws, nullptr) != GM_OK || cudaEventCreateWithFlags(&S.done_ev, cudaEventDisableTiming) !=
                                                         cudaSuccess) {
            for (auto &T : srv->eng.slots) {
                workspace_free(ctx, T.ws);
                if (T.done_ev) cudaEventDestroy(T.done_ev);
            }
            delete srv;
            return nullptr;
        }
    }
    int64_t cap = kMaxSlotQueries;
    if (ctx->budget) {
        const int64_t left = (int64_t)ctx->budget - (int64_t)ctx->bytes_images - (int64_t)ctx->bytes_work;
        cap = std::min<int64_t>(cap, std::max<int64_t>(left, 0) / n / kBytesPerQuery);
    }
    srv->sched = new Scheduler<GpuEngine>(srv->eng, n, cap, kMaxBatchPairs, kMaxPending);
    return srv;
}

void server_stop(Server *srv)
{
    if (!srv) return;
    srv->sched->stop();
    delete srv->sched;
    for (auto &S : srv->eng.slots) {
        workspace_free(srv->eng.ctx, S.ws);
        if (S.done_ev) cudaEventDestroy(S.done_ev);
    }
    delete srv;
}

gm_status server_submit(Server *srv, const gm_pair &pair, uint64_t *ticket)
{
    const gm_status st = srv->sched->submit(pair, ticket);
    if (st == GM_ERR_BUDGET) return fail(st, "gm_submit: the request does not fit the device-memory budget");
    if (st == GM_ERR_BUSY) return fail(st, "gm_submit: the serving queue is full");
    if (st != GM_OK) return st;   // message set by prepare_pair
    return GM_OK;
}

gm_status server_poll(Server *srv, uint64_t ticket, int32_t *matches, int64_t cap, int64_t *n, int32_t timeout_ms,
                      double *latency_us)
{
    const gm_status st = srv->sched->poll(ticket, matches, cap, n, timeout_ms, latency_us);
    switch (st) {
    case GM_OK: return GM_OK;
    case GM_ERR_TIMEOUT: return fail(st, "gm_poll: request %llu not done yet", (unsigned long long)ticket);
    case GM_ERR_NOT_FOUND: return fail(st, "gm_poll: unknown ticket %llu", (unsigned long long)ticket);
    case GM_ERR_NOMEM: return fail(st, "gm_poll: %lld matches exceed cap %lld", (long long)*n, (long long)cap);
    default: return fail(st, "gm_poll: request %llu failed (%d)", (unsigned long long)ticket, (int)st);
    }
}

void server_drain(Server *srv)
{
    for (auto &S : srv->eng.slots)
        if (S.ws.stream) cudaStreamSynchronize(S.ws.stream);
}

gm_status server_stats(Server *srv, gm_serving_stats *out)
{
    const SchedStats s = srv->sched->stats();
    out->submitted = s.submitted;
    out->completed = s.completed;
    out->failed = s.failed;
    out->batches = s.batches;
    out->max_batch_pairs = s.max_batch;
    out->peak_inflight_batches = s.peak_inflight;
    out->rejected_budget = s.rejected_budget;
    out->rejected_busy = s.rejected_busy;
    return GM_OK;
}

void server_wait_idle(Server *srv) { srv->sched->drain(); }

void server_referenced(Server *srv, std::unordered_set<int32_t> &ids) { srv->sched->referenced_images(ids); }

}  // namespace gm
