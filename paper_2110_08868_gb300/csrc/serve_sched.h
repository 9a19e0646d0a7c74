// Job scheduler of the reconstruction server (pure C++17, no CUDA).
//
// Jobs are admitted in arrival order (FIFO, no overtaking) while two resources allow:
// device bytes (each job declares its footprint; the sum over admitted jobs stays
// within the budget) and slots (at most max_active jobs on the device at once). An
// admitted job runs on a worker thread of its own; its device work is the run
// function given to the scheduler, which for the server creates the job's context on
// a stream of its own, so the admitted jobs' kernels overlap on the device. When a
// job finishes, its bytes and slot are released and the queue is admitted again, so
// jobs that arrived while others were running start as soon as room frees up.
//
// A finished job keeps its record (outputs, return code, times) until take() hands
// it to the caller. Times are seconds since the scheduler was constructed: arrival
// (submit), admission, completion; latency = completion - arrival.
//
// The device work is injected, so this file is tested on the CPU with a fake run
// function.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include "sdot.h"

namespace sdot {
namespace serve {

template <class Payload>
class Scheduler {
public:
    // run(payload) performs the job's device work and returns SDOT_OK or an error code
    using RunFn = std::function<int(Payload&)>;

    struct Info {
        size_t budget, used, peak_used;
        int max_active, active, peak_active;
        int64_t queued, finished, submitted;
    };

    Scheduler(size_t budget, int max_active, RunFn run)
        : budget_(budget), max_active_(max_active < 1 ? 1 : max_active), run_(std::move(run)),
          t0_(std::chrono::steady_clock::now()) {}

    Scheduler(const Scheduler&) = delete;
    Scheduler& operator=(const Scheduler&) = delete;

    // Drops the jobs still queued and waits for the running ones.
    ~Scheduler() {
        std::unique_lock<std::mutex> lk(mu_);
        stopping_ = true;
        for (int64_t id : queue_) jobs_.erase(id);
        queue_.clear();
        cv_.wait(lk, [&] { return active_ == 0; });
        reap_locked();
        std::vector<std::thread> rest;
        for (auto& kv : threads_) rest.push_back(std::move(kv.second));
        threads_.clear();
        lk.unlock();
        for (auto& t : rest)
            if (t.joinable()) t.join();
    }

    // Queue a job; *id receives its identifier. A job that could never fit the budget
    // is refused with SDOT_ERR_OOM.
    int submit(Payload&& p, size_t footprint, int64_t* id) {
        if (!id) return SDOT_ERR_ARG;
        std::lock_guard<std::mutex> lk(mu_);
        if (stopping_) return SDOT_ERR_ARG;
        if (footprint > budget_) return SDOT_ERR_OOM;
        const int64_t jid = next_id_++;
        Record& r = jobs_[jid];
        r.footprint = footprint;
        r.state = SDOT_JOB_QUEUED;
        r.rc = SDOT_OK;
        r.t_submit = now();
        r.t_admit = r.t_done = -1.0;
        r.payload = std::move(p);
        queue_.push_back(jid);
        submitted_++;
        *id = jid;
        admit_locked();
        return SDOT_OK;
    }

    int state(int64_t id, int* st) const {
        if (!st) return SDOT_ERR_ARG;
        std::lock_guard<std::mutex> lk(mu_);
        auto it = jobs_.find(id);
        if (it == jobs_.end()) return SDOT_ERR_ARG;
        *st = it->second.state;
        return SDOT_OK;
    }

    // Wait until job id has finished (state DONE or FAILED) or timeout_s seconds have
    // passed (timeout_s < 0: no limit). Returns SDOT_ERR_TIMEOUT if it has not finished.
    int wait(int64_t id, double timeout_s, int* st) {
        std::unique_lock<std::mutex> lk(mu_);
        auto finished = [&] {
            auto it = jobs_.find(id);
            return it == jobs_.end() || it->second.state >= SDOT_JOB_DONE;
        };
        if (jobs_.find(id) == jobs_.end()) return SDOT_ERR_ARG;
        if (timeout_s < 0) {
            cv_.wait(lk, finished);
        } else {
            cv_.wait_for(lk, std::chrono::duration<double>(timeout_s), finished);
        }
        auto it = jobs_.find(id);
        if (it == jobs_.end()) return SDOT_ERR_ARG;
        if (st) *st = it->second.state;
        return it->second.state >= SDOT_JOB_DONE ? SDOT_OK : SDOT_ERR_TIMEOUT;
    }

    // Hand a finished job to the caller and forget it: *out receives the payload,
    // *rc the job's return code, t[0..2] its arrival, admission and completion times.
    // SDOT_ERR_NOT_READY while it is queued or running.
    int take(int64_t id, Payload* out, int* rc, double t[3]) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = jobs_.find(id);
        if (it == jobs_.end()) return SDOT_ERR_ARG;
        Record& r = it->second;
        if (r.state < SDOT_JOB_DONE) return SDOT_ERR_NOT_READY;
        if (out) *out = std::move(r.payload);
        if (rc) *rc = r.rc;
        if (t) {
            t[0] = r.t_submit;
            t[1] = r.t_admit;
            t[2] = r.t_done;
        }
        jobs_.erase(it);
        reap_locked();
        return SDOT_OK;
    }

    Info info() const {
        std::lock_guard<std::mutex> lk(mu_);
        Info f;
        f.budget = budget_;
        f.used = used_;
        f.peak_used = peak_used_;
        f.max_active = max_active_;
        f.active = active_;
        f.peak_active = peak_active_;
        f.queued = (int64_t)queue_.size();
        f.finished = finished_;
        f.submitted = submitted_;
        return f;
    }

private:
    struct Record {
        size_t footprint = 0;
        int state = SDOT_JOB_QUEUED;
        int rc = SDOT_OK;
        double t_submit = 0, t_admit = 0, t_done = 0;
        Payload payload{};
    };

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0_).count();
    }

    // admit from the head of the queue while the head fits (no overtaking)
    void admit_locked() {
        reap_locked();
        while (!stopping_ && !queue_.empty() && active_ < max_active_) {
            const int64_t jid = queue_.front();
            Record& r = jobs_[jid];
            if (used_ + r.footprint > budget_) break;
            queue_.pop_front();
            used_ += r.footprint;
            active_++;
            if (used_ > peak_used_) peak_used_ = used_;
            if (active_ > peak_active_) peak_active_ = active_;
            r.state = SDOT_JOB_RUNNING;
            r.t_admit = now();
            threads_[jid] = std::thread(&Scheduler::worker, this, jid);
        }
    }

    // join the threads of jobs that have finished (they no longer touch the lock)
    void reap_locked() {
        for (int64_t jid : done_threads_) {
            auto it = threads_.find(jid);
            if (it != threads_.end()) {
                if (it->second.joinable()) it->second.join();
                threads_.erase(it);
            }
        }
        done_threads_.clear();
    }

    void worker(int64_t jid) {
        Payload* p = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu_);
            p = &jobs_[jid].payload;  // map nodes are stable; the record stays until take()
        }
        int rc = SDOT_ERR_ARG;
        try {
            rc = run_(*p);
        } catch (...) {
            rc = SDOT_ERR_ARG;
        }
        std::lock_guard<std::mutex> lk(mu_);
        Record& r = jobs_[jid];
        r.rc = rc;
        r.state = rc == SDOT_OK ? SDOT_JOB_DONE : SDOT_JOB_FAILED;
        r.t_done = now();
        used_ -= r.footprint;
        active_--;
        finished_++;
        done_threads_.push_back(jid);
        // the thread of this job is joined later by another caller; admit from here
        // without reaping (a thread cannot join itself)
        std::vector<int64_t> keep;
        keep.swap(done_threads_);
        admit_locked();
        done_threads_.swap(keep);
        cv_.notify_all();
    }

    const size_t budget_;
    const int max_active_;
    RunFn run_;
    const std::chrono::steady_clock::time_point t0_;

    mutable std::mutex mu_;
    std::condition_variable cv_;
    std::map<int64_t, Record> jobs_;
    std::deque<int64_t> queue_;
    std::map<int64_t, std::thread> threads_;
    std::vector<int64_t> done_threads_;
    int64_t next_id_ = 1;
    size_t used_ = 0, peak_used_ = 0;
    int active_ = 0, peak_active_ = 0;
    int64_t finished_ = 0, submitted_ = 0;
    bool stopping_ = false;
};

// Gathers requests of concurrent callers into batches for one worker thread. A caller
// blocks in submit() until the batch holding its request has run. The worker takes
// the first pending request, waits up to `window` for more (or until as many are
// pending as callers are active), hands up to max_batch requests to run_batch (which
// fills in their results), and wakes their callers. fini runs on the worker thread
// when it exits. The batch composition never changes what run_batch computes for a
// request, only when it runs.
template <class Req>
class Batcher {
public:
    using RunFn = std::function<void(std::vector<Req*>&)>;
    using FiniFn = std::function<void()>;

    struct Stats {
        int64_t batches, requests;
        int max_batch_seen;
    };

    Batcher(std::chrono::microseconds window, int max_batch, RunFn run, FiniFn fini = nullptr)
        : window_(window), max_batch_(max_batch < 1 ? 1 : max_batch), run_(std::move(run)),
          fini_(std::move(fini)) {
        th_ = std::thread(&Batcher::loop, this);
    }

    Batcher(const Batcher&) = delete;
    Batcher& operator=(const Batcher&) = delete;

    // Stops the worker; no caller may be inside submit() any more.
    ~Batcher() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        th_.join();
    }

    // callers that may submit soon (the window ends early once all of them wait)
    void add_active(int delta) {
        {
            std::lock_guard<std::mutex> lk(mu_);
            active_ += delta;
        }
        cv_.notify_all();
    }

    void submit(Req* r) {
        Slot q;
        q.req = r;
        std::unique_lock<std::mutex> lk(mu_);
        pending_.push_back(&q);
        cv_.notify_all();
        done_cv_.wait(lk, [&] { return q.done; });
    }

    Stats stats() const {
        std::lock_guard<std::mutex> lk(mu_);
        return Stats{batches_, requests_, max_seen_};
    }

private:
    struct Slot {
        Req* req = nullptr;
        bool done = false;
    };

    void loop() {
        std::unique_lock<std::mutex> lk(mu_);
        while (true) {
            cv_.wait(lk, [&] { return stop_ || !pending_.empty(); });
            if (pending_.empty()) break;  // stop requested, nothing left
            cv_.wait_until(lk, std::chrono::steady_clock::now() + window_, [&] {
                return stop_ || (int)pending_.size() >= active_;
            });
            std::vector<Slot*> slots;
            while (!pending_.empty() && (int)slots.size() < max_batch_) {
                slots.push_back(pending_.front());
                pending_.pop_front();
            }
            lk.unlock();
            std::vector<Req*> reqs;
            for (Slot* q : slots) reqs.push_back(q->req);
            run_(reqs);
            lk.lock();
            batches_++;
            requests_ += (int64_t)slots.size();
            if ((int)slots.size() > max_seen_) max_seen_ = (int)slots.size();
            for (Slot* q : slots) q->done = true;
            done_cv_.notify_all();
        }
        lk.unlock();
        if (fini_) fini_();
    }

    const std::chrono::microseconds window_;
    const int max_batch_;
    RunFn run_;
    FiniFn fini_;
    std::thread th_;
    mutable std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::deque<Slot*> pending_;
    int active_ = 0;
    bool stop_ = false;
    int64_t batches_ = 0, requests_ = 0;
    int max_seen_ = 0;
};

}  // namespace serve
}  // namespace sdot
