// CPU test of the server's job scheduler (serve_sched.h) with a fake device: the run
// function sleeps and records how many jobs and bytes were on the "device" at once.
// Built and run by tests/test_serve_sched.py; prints one line per check and exits
// non-zero on the first failure.
#include <stdio.h>
#include <stdlib.h>

#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "serve_sched.h"

using sdot::serve::Batcher;
using sdot::serve::Scheduler;

namespace {

struct Fake {
    int sleep_ms = 20;
    int fail = 0;       // run returns this code
    size_t bytes = 0;   // footprint, for the concurrency record
    int order = -1;     // start order, written by run
};

std::atomic<int> g_running{0}, g_peak_running{0}, g_started{0};
std::atomic<size_t> g_bytes{0}, g_peak_bytes{0};

int fake_run(Fake& f) {
    f.order = g_started.fetch_add(1);
    int r = ++g_running;
    size_t b = (g_bytes += f.bytes);
    int pr = g_peak_running.load();
    while (r > pr && !g_peak_running.compare_exchange_weak(pr, r)) {}
    size_t pb = g_peak_bytes.load();
    while (b > pb && !g_peak_bytes.compare_exchange_weak(pb, b)) {}
    std::this_thread::sleep_for(std::chrono::milliseconds(f.sleep_ms));
    g_bytes -= f.bytes;
    --g_running;
    return f.fail;
}

void reset() {
    g_running = 0;
    g_peak_running = 0;
    g_started = 0;
    g_bytes = 0;
    g_peak_bytes = 0;
}

int g_fail = 0;
void check(bool ok, const char* what) {
    printf("%s %s\n", ok ? "ok  " : "FAIL", what);
    if (!ok) g_fail = 1;
}

Fake job(size_t bytes, int ms, int fail = 0) {
    Fake f;
    f.bytes = bytes;
    f.sleep_ms = ms;
    f.fail = fail;
    return f;
}

}  // namespace

int main() {
    // 1. the byte budget bounds what runs at once; every job completes
    {
        reset();
        Scheduler<Fake> s(100, 8, fake_run);
        std::vector<int64_t> ids;
        for (int t = 0; t < 10; t++) {
            int64_t id = 0;
            check(s.submit(job(40, 20), 40, &id) == SDOT_OK, "submit within budget");
            ids.push_back(id);
        }
        for (int64_t id : ids) {
            int st = -1;
            check(s.wait(id, 10.0, &st) == SDOT_OK && st == SDOT_JOB_DONE, "job done");
        }
        auto f = s.info();
        check(f.peak_used <= 100 && f.peak_active <= 2, "budget 100, footprint 40: <= 2 at once");
        check(g_peak_bytes.load() <= 100 && g_peak_running.load() <= 2, "device view agrees");
        check(f.peak_active == 2, "two jobs did overlap");
        check(f.used == 0 && f.active == 0 && f.finished == 10, "resources released");
    }
    // 2. slots bound the concurrency when bytes do not
    {
        reset();
        Scheduler<Fake> s(1000, 3, fake_run);
        std::vector<int64_t> ids(12);
        for (auto& id : ids) s.submit(job(1, 15), 1, &id);
        for (int64_t id : ids) s.wait(id, 10.0, nullptr);
        check(s.info().peak_active == 3 && g_peak_running.load() == 3, "3 slots: 3 at once");
    }
    // 3. FIFO without overtaking: a large job at the head makes later small jobs wait
    {
        reset();
        Scheduler<Fake> s(100, 8, fake_run);
        int64_t a, b, c, d;
        s.submit(job(60, 60), 60, &a);  // runs
        s.submit(job(60, 10), 60, &b);  // waits for a
        s.submit(job(10, 10), 10, &c);  // fits now, but must not overtake b
        s.submit(job(10, 10), 10, &d);
        for (int64_t id : {a, b, c, d}) s.wait(id, 10.0, nullptr);
        Fake fa, fb, fc, fd;
        double ta[3], tb[3], tc[3], td[3];
        int rc;
        s.take(a, &fa, &rc, ta);
        s.take(b, &fb, &rc, tb);
        s.take(c, &fc, &rc, tc);
        s.take(d, &fd, &rc, td);
        check(fa.order == 0, "the head job started alone");
        check(tb[1] >= ta[2], "b admitted only after a finished");
        check(tc[1] >= ta[2] && td[1] >= ta[2], "c and d did not overtake b");
        check(tc[1] >= tb[1] && td[1] >= tc[1], "admission times non-decreasing");
        check(ta[0] <= tb[0] && ta[0] <= ta[1] && ta[1] <= ta[2], "arrival <= admission <= done");
    }
    // 4. a job larger than the budget is refused at submission
    {
        reset();
        Scheduler<Fake> s(100, 8, fake_run);
        int64_t id = 0;
        check(s.submit(job(101, 1), 101, &id) == SDOT_ERR_OOM, "oversize job refused");
        check(s.info().submitted == 0, "nothing queued");
    }
    // 5. a failing job reports its code; the others are unaffected
    {
        reset();
        Scheduler<Fake> s(100, 4, fake_run);
        int64_t bad, good;
        s.submit(job(10, 5, SDOT_ERR_NO_DESCENT), 10, &bad);
        s.submit(job(10, 5), 10, &good);
        int st = -1;
        s.wait(bad, 10.0, &st);
        check(st == SDOT_JOB_FAILED, "failed state");
        int rc = 0;
        check(s.take(bad, nullptr, &rc, nullptr) == SDOT_OK && rc == SDOT_ERR_NO_DESCENT,
              "error code kept");
        s.wait(good, 10.0, &st);
        check(st == SDOT_JOB_DONE, "other job done");
    }
    // 6. waits with a limit, results before completion, unknown ids
    {
        reset();
        Scheduler<Fake> s(100, 1, fake_run);
        int64_t slow, next;
        s.submit(job(10, 300), 10, &slow);
        s.submit(job(10, 5), 10, &next);
        int st = -1;
        check(s.wait(slow, 0.01, &st) == SDOT_ERR_TIMEOUT && st == SDOT_JOB_RUNNING,
              "timed wait on a running job");
        check(s.state(next, &st) == SDOT_OK && st == SDOT_JOB_QUEUED, "second job queued (1 slot)");
        check(s.take(slow, nullptr, nullptr, nullptr) == SDOT_ERR_NOT_READY, "take before done");
        check(s.take(12345, nullptr, nullptr, nullptr) == SDOT_ERR_ARG, "unknown id");
        s.wait(next, 10.0, &st);
        check(st == SDOT_JOB_DONE, "queued job ran after the slot freed");
    }
    // 7. destruction with running and queued jobs: running ones finish, queued are dropped
    {
        reset();
        {
            Scheduler<Fake> s(100, 1, fake_run);
            int64_t id;
            s.submit(job(10, 50), 10, &id);
            for (int t = 0; t < 5; t++) s.submit(job(10, 50), 10, &id);
        }
        check(g_started.load() == 1 && g_running.load() == 0, "destructor waits, drops the queue");
    }
    // 8. many submitters at once (thread safety of submit/wait/take)
    {
        reset();
        Scheduler<Fake> s(50, 4, fake_run);
        std::atomic<int> ok{0};
        std::vector<std::thread> th;
        for (int t = 0; t < 8; t++)
            th.emplace_back([&] {
                for (int u = 0; u < 8; u++) {
                    int64_t id;
                    if (s.submit(job(10, 2), 10, &id) != SDOT_OK) continue;
                    int st;
                    if (s.wait(id, 20.0, &st) == SDOT_OK && st == SDOT_JOB_DONE &&
                        s.take(id, nullptr, nullptr, nullptr) == SDOT_OK)
                        ok++;
                }
            });
        for (auto& t : th) t.join();
        auto f = s.info();
        check(ok.load() == 64 && f.finished == 64 && f.peak_used <= 50 && f.peak_active <= 4,
              "64 jobs from 8 threads");
    }
    // 9. batcher: every request gets its own result; concurrent requests share batches
    {
        struct R {
            int in = 0, out = 0, batch = 0;
        };
        Batcher<R> b(std::chrono::microseconds(2000), 4, [](std::vector<R*>& rs) {
            for (R* r : rs) {
                r->out = 2 * r->in;
                r->batch = (int)rs.size();
            }
            std::this_thread::sleep_for(std::chrono::milliseconds(1));
        });
        b.add_active(8);
        std::atomic<int> bad{0}, shared{0};
        std::vector<std::thread> th;
        for (int t = 0; t < 8; t++)
            th.emplace_back([&, t] {
                for (int u = 0; u < 25; u++) {
                    R r;
                    r.in = 1000 * t + u;
                    b.submit(&r);
                    if (r.out != 2 * r.in) bad++;
                    if (r.batch > 1) shared++;
                }
                b.add_active(-1);
            });
        for (auto& t : th) t.join();
        auto st = b.stats();
        check(bad.load() == 0, "batcher: each request gets its own result");
        check(st.requests == 200, "batcher: every request ran once");
        check(st.max_batch_seen <= 4, "batcher: batches capped at max_batch");
        check(shared.load() > 0 && st.batches < 200, "batcher: concurrent requests share batches");
    }
    // 10. the window: a lone active caller runs at once; with another caller active
    //     (but silent) the batch waits the window out
    {
        struct R {
            int x = 0;
        };
        Batcher<R> b(std::chrono::milliseconds(60), 8, [](std::vector<R*>&) {});
        b.add_active(1);
        R r;
        auto t0 = std::chrono::steady_clock::now();
        b.submit(&r);
        double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        check(dt < 0.04, "batcher: a lone caller does not wait for the window");
        b.add_active(1);
        t0 = std::chrono::steady_clock::now();
        b.submit(&r);
        dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        check(dt >= 0.05, "batcher: waits the window for the other active caller");
        b.add_active(-2);
    }
    // 11. fini runs on the worker thread when the batcher is destroyed
    {
        std::atomic<bool> fini_ran{false};
        std::thread::id worker_id, fini_id;
        {
            struct R {
                int x = 0;
            };
            Batcher<R> b(
                std::chrono::microseconds(100), 2,
                [&](std::vector<R*>&) { worker_id = std::this_thread::get_id(); },
                [&] {
                    fini_id = std::this_thread::get_id();
                    fini_ran = true;
                });
            R r;
            b.submit(&r);
        }
        check(fini_ran.load() && fini_id == worker_id, "batcher: fini on the worker thread");
    }
    return g_fail;
}
