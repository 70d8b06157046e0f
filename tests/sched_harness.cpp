// sched_harness.cpp -- host-side tests of the serving scheduler (gm_sched.h) with a stub engine: no GPU.
//
// The stub engine answers each request with rows derived from its pair (so a result can be checked against the
// request alone), completes a batch after a configurable number of polls, and injects failures on request:
// pair.img_a < 0 is refused at submission (cost error), pair.img_b == 99 makes the batch's launch fail,
// pair.img_b == 98 never completes until the test releases the engine.  Each mode prints one JSON object.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../paper_1512_06235_gb300/csrc/gm_sched.h"

namespace {

struct StubEngine {
    std::atomic<bool> release{true};
    std::atomic<int> launches{0};
    std::atomic<int64_t> capacity{1 << 30};   // what slot_capacity() reports (the budget share of the moment)
    std::atomic<int64_t> max_multi_cost{0};   // largest total cost of a batch of two or more requests
    std::vector<std::vector<gm::SchedRequest *>> inflight;
    std::vector<int> polls_left;
    explicit StubEngine(int slots) : inflight(slots), polls_left(slots, 0) {}

    int64_t cost(const gm_pair &p, gm_status *err)
    {
        if (p.img_a < 0) {
            *err = GM_ERR_NOT_FOUND;
            return -1;
        }
        return 1 + (p.img_a % 7);
    }
    int64_t slot_capacity() { return capacity.load(); }
    gm_status launch(int s, std::vector<gm::SchedRequest *> &batch)
    {
        ++launches;
        int64_t c = 0;
        for (auto *r : batch) c += r->cost;
        if (batch.size() > 1 && c > max_multi_cost) max_multi_cost = c;
        for (auto *r : batch)
            if (r->pair.img_b == 99) return GM_ERR_CUDA;
        inflight[s] = batch;
        polls_left[s] = 2;
        return GM_OK;
    }
    bool done(int s)
    {
        for (auto *r : inflight[s])
            if (r->pair.img_b == 98 && !release) return false;
        return --polls_left[s] <= 0;
    }
    void collect(int s, std::vector<gm::SchedRequest *> &batch)
    {
        for (auto *r : batch) {
            if (r->status != GM_OK) continue;
            r->rows = {r->pair.img_a, r->pair.img_b, r->pair.ratio_num, r->pair.ratio_den};
        }
        inflight[s].clear();
    }
};

gm_pair make(int a, int b, int p = 4, int q = 5)
{
    gm_pair g{};
    g.img_a = a;
    g.img_b = b;
    g.band_px = 4.0f;
    g.ratio_num = (uint16_t)p;
    g.ratio_den = (uint16_t)q;
    return g;
}

bool check_rows(gm::Scheduler<StubEngine> &S, uint64_t t, const gm_pair &p, int32_t timeout_ms = 5000)
{
    int32_t out[8];
    int64_t n = 0;
    if (S.poll(t, out, 4, &n, timeout_ms, nullptr) != GM_OK || n != 2) return false;
    return out[0] == p.img_a && out[1] == p.img_b && out[2] == p.ratio_num && out[3] == p.ratio_den;
}

int mix()   // continuous batching: every result equals the request alone; batches respect the capacity
{
    StubEngine E(2);
    gm::Scheduler<StubEngine> S(E, 2, 10, 64, 1 << 16);
    const int n = 2000;
    std::vector<std::thread> th;
    std::atomic<int> bad{0};
    for (int w = 0; w < 4; ++w)
        th.emplace_back([&, w] {
            for (int k = 0; k < n / 4; ++k) {
                const gm_pair p = make(w * 1000 + k, k % 50, 1 + k % 3, 5);
                uint64_t t = 0;
                if (S.submit(p, &t) != GM_OK || !check_rows(S, t, p)) ++bad;
            }
        });
    for (auto &t : th) t.join();
    const gm::SchedStats st = S.stats();
    std::printf("{\"bad\": %d, \"completed\": %lld, \"batches\": %lld, \"max_batch\": %lld}\n", bad.load(),
                (long long)st.completed, (long long)st.batches, (long long)st.max_batch);
    return 0;
}

int faults()
{
    StubEngine E(1);
    gm::Scheduler<StubEngine> S(E, 1, 10, 64, 4);
    uint64_t t = 0;
    const gm_status unknown = S.submit(make(-1, 0), &t);          // refused at submission
    const gm_status fits = S.submit(make(20, 0), &t);             // cost 7 fits a slot of 10
    gm_status budget = GM_OK;
    {
        gm::Scheduler<StubEngine> small(E, 1, 3, 64, 4);
        budget = small.submit(make(6, 0), &t);                     // cost 7 > capacity 3
    }
    uint64_t tf = 0;
    S.submit(make(1, 99), &tf);                                    // its batch's launch fails
    int32_t out[8];
    int64_t n = 0;
    const gm_status launch_fail = S.poll(tf, out, 4, &n, 5000, nullptr);
    // a batch that does not complete: poll times out, then succeeds once released
    E.release = false;
    uint64_t ts = 0;
    S.submit(make(2, 98), &ts);
    const gm_status timeout = S.poll(ts, out, 4, &n, 20, nullptr);
    // the queue is bounded: with the engine held, the fourth queued request is refused
    std::vector<gm_status> q;
    for (int k = 0; k < 8; ++k) {
        uint64_t tk = 0;
        q.push_back(S.submit(make(3 + k, 98), &tk));
    }
    int busy = 0;
    for (auto s : q) busy += s == GM_ERR_BUSY;
    E.release = true;
    const gm_status after = S.poll(ts, out, 4, &n, 5000, nullptr);
    const gm::SchedStats st = S.stats();
    std::printf("{\"unknown\": %d, \"fits\": %d, \"budget\": %d, \"launch_fail\": %d, \"timeout\": %d, \"busy\": %d, "
                "\"after_release\": %d, \"rejected_budget\": %lld, \"rejected_busy\": %lld, \"failed\": %lld}\n",
                (int)unknown, (int)fits, (int)budget, (int)launch_fail, (int)timeout, busy, (int)after,
                (long long)st.rejected_budget, (long long)st.rejected_busy, (long long)st.failed);
    return 0;
}

int cancel()   // requests still queued when the scheduler stops end with GM_ERR_CANCELLED
{
    StubEngine E(1);
    E.release = false;
    std::vector<uint64_t> ts(6);
    gm::Scheduler<StubEngine> *S = new gm::Scheduler<StubEngine>(E, 1, 100, 1, 64);   // one request per batch
    for (int k = 0; k < 6; ++k) S->submit(make(k, 98), &ts[k]);   // the first is launched and held, five queue
    for (int w = 0; w < 1000 && E.launches.load() == 0; ++w)       // until the first batch is on the engine
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    std::thread stopper([&] {
        std::this_thread::sleep_for(std::chrono::milliseconds(50));
        E.release = true;   // the running batch may finish; the rest is cancelled by stop()
    });
    S->stop();
    stopper.join();
    int cancelled = 0, ok = 0, other = 0;
    for (uint64_t t : ts) {
        int32_t out[8];
        int64_t n = 0;
        const gm_status st = S->poll(t, out, 4, &n, 1000, nullptr);
        if (st == GM_ERR_CANCELLED) ++cancelled;
        else if (st == GM_OK) ++ok;
        else ++other;
    }
    uint64_t t = 0;
    const gm_status after_stop = S->submit(make(1, 1), &t);
    delete S;
    std::printf("{\"cancelled\": %d, \"ok\": %d, \"other\": %d, \"after_stop\": %d}\n", cancelled, ok, other,
                (int)after_stop);
    return 0;
}

int shrink()   // the engine's capacity of the moment bounds every batch; a larger request runs alone when idle
{
    StubEngine E(2);
    E.capacity = 4;   // below the construction capacity (10) and below the costliest requests (7)
    gm::Scheduler<StubEngine> S(E, 2, 10, 64, 1 << 16);
    const int n = 300;
    std::vector<std::thread> th;
    std::atomic<int> bad{0};
    for (int w = 0; w < 4; ++w)
        th.emplace_back([&, w] {   // every thread queues all its requests first, so batches can form
            std::vector<std::pair<uint64_t, gm_pair>> mine;
            for (int k = 0; k < n / 4; ++k) {
                const gm_pair p = make(w * 1000 + k, k % 50);
                uint64_t t = 0;
                if (S.submit(p, &t) != GM_OK) ++bad;
                else mine.emplace_back(t, p);
            }
            for (auto &tp : mine)
                if (!check_rows(S, tp.first, tp.second)) ++bad;
        });
    for (auto &t : th) t.join();
    const gm::SchedStats st = S.stats();
    std::printf("{\"bad\": %d, \"completed\": %lld, \"max_multi_cost\": %lld}\n", bad.load(),
                (long long)st.completed, (long long)E.max_multi_cost.load());
    return 0;
}

}  // namespace

int main(int argc, char **argv)
{
    const std::string mode = argc > 1 ? argv[1] : "";
    if (mode == "mix") return mix();
    if (mode == "faults") return faults();
    if (mode == "cancel") return cancel();
    if (mode == "shrink") return shrink();
    std::fprintf(stderr, "usage: sched_harness mix|faults|cancel|shrink\n");
    return 2;
}
