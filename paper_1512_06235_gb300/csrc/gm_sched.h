// gm_sched.h -- continuous-batching scheduler of the serving loop (pure C++17, no CUDA).
//
// Requests (one image pair each) are queued by submit(); a scheduler thread admits queued requests, in arrival
// order, into the next free batch slot while the slot's capacity allows (capacity = queries, i.e. the device
// workspace that the memory budget leaves per slot), launches the batch through the engine and goes on admitting
// into other slots while earlier batches run, so requests that arrive while the device is busy join the next
// batch and overlap with the running ones.  Completed batches are collected in any order.  Every wait is bounded:
// the engine is polled (never blocked on), and poll() takes a timeout.
//
// Admission uses the smaller of the capacity given at construction (which also bounds what submit() accepts) and
// the engine's current slot capacity, read before every round of admissions (the budget left for work buffers
// changes as images are put and evicted).  When nothing is in flight, the first queued request is admitted even if
// it exceeds the current capacity, so that the queue never stalls: the engine then runs it or fails it.
//
// Engine requirements (duck-typed):
//   int64_t cost(const gm_pair&, gm_status* err);           // queries the request needs, or -1 (err set)
//   int64_t slot_capacity();                                  // queries one batch may take now
//   gm_status launch(int slot, std::vector<Request*>& batch); // enqueue; on error every request gets the status
//   bool done(int slot);                                      // non-blocking completion test
//   void collect(int slot, std::vector<Request*>& batch);     // fill rows / status of each request
#pragma once
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/geomatch.h"

namespace gm {

struct SchedRequest {
    uint64_t ticket = 0;
    gm_pair pair{};
    int64_t cost = 0;
    gm_status status = GM_OK;
    bool done = false;
    std::vector<int32_t> rows;   // (i, j) pairs, sorted by i
    std::chrono::steady_clock::time_point t_submit, t_done;
};

struct SchedStats {
    int64_t submitted = 0, completed = 0, failed = 0, batches = 0, max_batch = 0, peak_inflight = 0;
    int64_t rejected_budget = 0, rejected_busy = 0;
};

template <class Engine>
class Scheduler {
public:
    using Request = SchedRequest;

    Scheduler(Engine &eng, int n_slots, int64_t slot_capacity, int max_batch_pairs, size_t max_pending)
        : eng_(eng), slots_(n_slots), capacity_(slot_capacity), max_batch_pairs_(max_batch_pairs),
          max_pending_(max_pending)
    {
        th_ = std::thread([this] { loop(); });
    }

    ~Scheduler() { stop(); }

    gm_status submit(const gm_pair &pair, uint64_t *ticket)
    {
        gm_status err = GM_OK;
        const int64_t cost = eng_.cost(pair, &err);
        std::lock_guard<std::mutex> lk(mu_);
        if (cost < 0) return err;
        if (stop_) return GM_ERR_CANCELLED;
        if (cost > capacity_) {
            ++stats_.rejected_budget;
            return GM_ERR_BUDGET;
        }
        if (pending_.size() >= max_pending_) {
            ++stats_.rejected_busy;
            return GM_ERR_BUSY;
        }
        auto r = std::make_shared<Request>();
        r->ticket = next_ticket_++;
        r->pair = pair;
        r->cost = cost;
        r->t_submit = std::chrono::steady_clock::now();
        table_[r->ticket] = r;
        pending_.push_back(r);
        ++stats_.submitted;
        *ticket = r->ticket;
        cv_work_.notify_one();
        return GM_OK;
    }

    gm_status poll(uint64_t ticket, int32_t *out, int64_t cap, int64_t *n, int32_t timeout_ms, double *latency_us)
    {
        std::unique_lock<std::mutex> lk(mu_);
        auto it = table_.find(ticket);
        if (it == table_.end()) return GM_ERR_NOT_FOUND;
        std::shared_ptr<Request> r = it->second;
        if (!r->done) {
            if (timeout_ms == 0) return GM_ERR_TIMEOUT;
            auto pred = [&] { return r->done; };
            if (timeout_ms < 0) cv_done_.wait(lk, pred);
            else if (!cv_done_.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return GM_ERR_TIMEOUT;
        }
        *n = (int64_t)(r->rows.size() / 2);
        if (latency_us)
            *latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
        if (r->status != GM_OK) {
            table_.erase(ticket);
            return r->status;
        }
        if (*n > cap) return GM_ERR_NOMEM;
        if (*n > 0) std::memcpy(out, r->rows.data(), sizeof(int32_t) * r->rows.size());
        table_.erase(ticket);
        return GM_OK;
    }

    // The image ids of every request not yet finished (queued, or taken into a batch): images that must stay
    // resident.  Never blocks on the engine (the scheduler holds mu_ only for its own bookkeeping).
    template <typename Set>
    void referenced_images(Set &ids)
    {
        std::lock_guard<std::mutex> lk(mu_);
        for (auto &r : pending_) { ids.insert(r->pair.img_a); ids.insert(r->pair.img_b); }
        for (auto &sl : slots_)
            for (auto &r : sl.reqs) { ids.insert(r->pair.img_a); ids.insert(r->pair.img_b); }
    }

    // Blocks until nothing is queued or in flight.
    void drain()
    {
        std::unique_lock<std::mutex> lk(mu_);
        cv_done_.wait(lk, [&] { return pending_.empty() && inflight_ == 0; });
    }

    void stop()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (stop_ && !th_.joinable()) return;
            stop_ = true;
            cv_work_.notify_all();
        }
        if (th_.joinable()) th_.join();
        std::lock_guard<std::mutex> lk(mu_);
        for (auto &r : pending_) finish(*r, GM_ERR_CANCELLED);
        pending_.clear();
        cv_done_.notify_all();
    }

    SchedStats stats()
    {
        std::lock_guard<std::mutex> lk(mu_);
        return stats_;
    }

private:
    struct Slot {
        bool busy = false;
        std::vector<std::shared_ptr<Request>> reqs;
        std::vector<Request *> raw;
    };

    void finish(Request &r, gm_status st)
    {
        r.status = st;
        r.done = true;
        r.t_done = std::chrono::steady_clock::now();
        if (st == GM_OK) ++stats_.completed;
        else ++stats_.failed;
    }

    void loop()
    {
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            // 1. collect finished batches
            bool progressed = false;
            for (size_t s = 0; s < slots_.size(); ++s) {
                Slot &sl = slots_[s];
                if (!sl.busy) continue;
                lk.unlock();
                const bool d = eng_.done((int)s);
                if (d) eng_.collect((int)s, sl.raw);
                lk.lock();
                if (!d) continue;
                for (auto &r : sl.reqs) finish(*r, r->status);
                sl.reqs.clear();
                sl.raw.clear();
                sl.busy = false;
                --inflight_;
                progressed = true;
            }
            if (progressed) cv_done_.notify_all();
            if (stop_ && inflight_ == 0) break;
            // 2. admit queued requests into free slots (continuous batching), against the capacity of now
            int64_t cap_now = capacity_;
            if (!pending_.empty()) {
                lk.unlock();
                const int64_t c = eng_.slot_capacity();
                lk.lock();
                cap_now = std::min(capacity_, c);
            }
            while (!stop_ && !pending_.empty()) {
                int free_slot = -1;
                for (size_t s = 0; s < slots_.size(); ++s)
                    if (!slots_[s].busy) { free_slot = (int)s; break; }
                if (free_slot < 0) break;
                Slot &sl = slots_[free_slot];
                int64_t used = 0;
                while (!pending_.empty() && (int)sl.reqs.size() < max_batch_pairs_ &&
                       (used + pending_.front()->cost <= cap_now || (sl.reqs.empty() && inflight_ == 0))) {
                    used += pending_.front()->cost;
                    sl.reqs.push_back(pending_.front());
                    pending_.pop_front();
                }
                if (sl.reqs.empty()) break;   // the next request waits for a running batch to finish
                for (auto &r : sl.reqs) sl.raw.push_back(r.get());
                sl.busy = true;
                ++inflight_;
                ++stats_.batches;
                stats_.max_batch = std::max<int64_t>(stats_.max_batch, (int64_t)sl.reqs.size());
                stats_.peak_inflight = std::max<int64_t>(stats_.peak_inflight, inflight_);
                lk.unlock();
                const gm_status st = eng_.launch(free_slot, sl.raw);
                lk.lock();
                if (st != GM_OK) {
                    for (auto &r : sl.reqs)
                        if (r->status == GM_OK) r->status = st;
                }
            }
            // 3. wait: briefly while batches run (the engine is polled), else until work arrives
            if (inflight_ > 0) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else if (!stop_) {
                cv_work_.wait_for(lk, std::chrono::milliseconds(50));
            }
        }
    }

    Engine &eng_;
    std::vector<Slot> slots_;
    int64_t capacity_;
    int max_batch_pairs_;
    size_t max_pending_;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::deque<std::shared_ptr<Request>> pending_;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> table_;
    uint64_t next_ticket_ = 1;
    int64_t inflight_ = 0;
    bool stop_ = false;
    SchedStats stats_;
    std::thread th_;
};

}  // namespace gm
