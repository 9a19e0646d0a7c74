// Reconstruction server (sdot_server_* in include/sdot.h).
//
// Jobs (one periodic box each, any N) are queued on submission with host copies of
// their inputs, admitted FIFO by device footprint and slot count (serve_sched.h), and
// each admitted job runs create + damped Newton + displacement on a non-blocking CUDA
// stream and worker thread of its own: the kernels of concurrent jobs overlap on the
// device, and each job's state stays resident until it finishes.
//
// Batched clipping (the default): a job's Laguerre evaluations go through the
// server's batcher. The batcher thread collects the requests of the running jobs
// (it waits a short window for the other jobs to ask too) and evaluates them together:
// each clipping pass is one persistent launch whose warps pull cells of all the
// batch's jobs from one shared work counter. The per-cell arithmetic and the per-job
// reductions are those of the single-box path, so a job's results do not depend on
// the other jobs in the batch.
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "serve_sched.h"

namespace sdot {
namespace {

struct JobPayload {
    std::vector<double> pos, mass;  // host copies of the inputs (mass empty: uniform)
    int64_t N = 0;
    double box[3] = {0, 0, 0};
    sdot_options opt{};
    double tol = 0;
    std::vector<double> disp, psi;  // outputs, caller order
    sdot_stats stats{};
    std::string err;
};

// most jobs evaluated in one batch
constexpr int MAX_BATCH = 64;
// how long the batcher waits for the other running jobs after the first request
constexpr auto BATCH_WINDOW = std::chrono::microseconds(200);

class Batcher {
public:
    explicit Batcher(int device) : device_(device) { th_ = std::thread(&Batcher::loop, this); }

    ~Batcher() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        th_.join();
    }

    void job_started() { active_++; }

    void job_finished() {
        active_--;
        cv_.notify_all();
    }

    // Called by a job's thread (hook of its context): wait until the job's earlier work
    // (and psi) is complete, queue the request, and wait for the batch result.
    int evaluate(DeviceState* d, const double* psi, int prec, EvalResult* r,
                 cudaStream_t job_stream) {
        cudaError_t e = cudaStreamSynchronize(job_stream);
        if (e != cudaSuccess) {
            set_error(std::string("batched evaluation: ") + cudaGetErrorString(e));
            return SDOT_ERR_CUDA;
        }
        Req q;
        q.d = d;
        q.psi = psi;
        q.prec = prec;
        q.r = r;
        std::unique_lock<std::mutex> lk(mu_);
        pending_.push_back(&q);
        cv_.notify_all();
        done_cv_.wait(lk, [&] { return q.done; });
        if (q.rc != SDOT_OK) set_error(q.err);
        return q.rc;
    }

    static int hook(void* user, DeviceState* d, const double* psi, int prec, EvalResult* r,
                    cudaStream_t s) {
        return static_cast<Batcher*>(user)->evaluate(d, psi, prec, r, s);
    }

private:
    struct Req {
        DeviceState* d = nullptr;
        const double* psi = nullptr;
        int prec = 0;
        EvalResult* r = nullptr;
        int rc = SDOT_OK;
        bool done = false;
        std::string err;
    };

    void loop() {
        cudaStream_t s = nullptr;
        BatchScratch* sc = nullptr;
        int init_rc = SDOT_OK;
        std::string init_err;
        if (cudaSetDevice(device_) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            init_rc = SDOT_ERR_CUDA;
            init_err = std::string("batcher: ") + cudaGetErrorString(cudaGetLastError());
        } else if ((init_rc = batch_scratch_create(MAX_BATCH, &sc)) != SDOT_OK) {
            init_err = sdot_last_error();
        }
        std::unique_lock<std::mutex> lk(mu_);
        while (true) {
            cv_.wait(lk, [&] { return stop_ || !pending_.empty(); });
            if (pending_.empty()) break;  // stop requested, nothing left
            // give the other running jobs a short window to join this batch
            cv_.wait_until(lk, std::chrono::steady_clock::now() + BATCH_WINDOW, [&] {
                return stop_ || (int)pending_.size() >= active_.load();
            });
            std::vector<Req*> batch;
            while (!pending_.empty() && (int)batch.size() < MAX_BATCH) {
                batch.push_back(pending_.front());
                pending_.pop_front();
            }
            lk.unlock();
            int rc = init_rc;
            std::string err = init_err;
            if (rc == SDOT_OK) {
                std::vector<DeviceState*> ds;
                std::vector<const double*> psis;
                std::vector<int> precs;
                std::vector<EvalResult> res(batch.size());
                for (Req* q : batch) {
                    ds.push_back(q->d);
                    psis.push_back(q->psi);
                    precs.push_back(q->prec);
                }
                rc = evaluate_cells_batch(ds.data(), psis.data(), precs.data(), res.data(),
                                          (int)batch.size(), sc, s);
                if (rc == SDOT_OK)
                    for (size_t t = 0; t < batch.size(); t++) *batch[t]->r = res[t];
                else
                    err = sdot_last_error();
            }
            lk.lock();
            for (Req* q : batch) {
                q->rc = rc;
                q->err = err;
                q->done = true;
            }
            done_cv_.notify_all();
        }
        lk.unlock();
        batch_scratch_destroy(sc);
        if (s) cudaStreamDestroy(s);
    }

    const int device_;
    std::thread th_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::deque<Req*> pending_;
    std::atomic<int> active_{0};
    bool stop_ = false;
};

bool host_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;  // not known to the runtime: plain host memory
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

// the device work of one job, on the calling worker thread (batcher: null for
// unbatched evaluations)
int run_job(int device, Batcher* batcher, JobPayload& j) {
    if (cudaSetDevice(device) != cudaSuccess) {
        j.err = std::string("server job: cudaSetDevice: ") + cudaGetErrorString(cudaGetLastError());
        return SDOT_ERR_CUDA;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        j.err = std::string("server job: stream: ") + cudaGetErrorString(cudaGetLastError());
        return SDOT_ERR_CUDA;
    }
    sdot_ctx* ctx = nullptr;
    int rc = create_context(j.pos.data(), j.mass.empty() ? nullptr : j.mass.data(), j.N, j.box,
                            &j.opt, s, &ctx);
    if (rc == SDOT_OK && batcher) {
        set_eval_hook(ctx, &Batcher::hook, batcher);
        batcher->job_started();
    }
    if (rc == SDOT_OK) rc = sdot_solve(ctx, j.tol, nullptr, &j.stats);
    if (ctx && batcher) batcher->job_finished();
    if (rc == SDOT_OK) {
        j.disp.resize((size_t)j.N * 3);
        rc = sdot_displacement(ctx, j.disp.data());
    }
    if (rc == SDOT_OK) {
        j.psi.resize((size_t)j.N);
        rc = sdot_get_psi(ctx, j.psi.data());
    }
    if (rc != SDOT_OK) {
        j.err = sdot_last_error();
        j.disp.clear();
        j.psi.clear();
    }
    sdot_destroy(ctx);
    cudaStreamDestroy(s);
    std::vector<double>().swap(j.pos);
    std::vector<double>().swap(j.mass);
    return rc;
}

}  // namespace
}  // namespace sdot

using namespace sdot;

struct sdot_server {
    int device = 0;
    // declared before the scheduler: destroyed after it, once no job can wait on it
    std::unique_ptr<Batcher> batcher;
    std::unique_ptr<serve::Scheduler<JobPayload>> sched;
};

extern "C" {

int sdot_server_default_options(sdot_server_options* o) {
    if (!o) return SDOT_ERR_ARG;
    o->hbm_budget = 0;
    o->max_active = 8;
    o->device = -1;
    o->batch_clip = 1;
    return SDOT_OK;
}

int sdot_server_footprint(int64_t N, const double box[3], const sdot_options* opt,
                          size_t* bytes) {
    set_error("");
    return context_footprint(N, box, opt, bytes);
}

int sdot_server_create(const sdot_server_options* opt, sdot_server** out) {
    set_error("");
    if (!out) {
        set_error("sdot_server_create: out is NULL");
        return SDOT_ERR_ARG;
    }
    *out = nullptr;
    sdot_server_options o;
    sdot_server_default_options(&o);
    if (opt) o = *opt;
    if (o.max_active < 1) {
        set_error("sdot_server_create: max_active must be >= 1");
        return SDOT_ERR_ARG;
    }
    int cur = 0, count = 0;
    SDOT_CUDA_TRY(cudaGetDevice(&cur));
    SDOT_CUDA_TRY(cudaGetDeviceCount(&count));
    const int dev = o.device < 0 ? cur : o.device;
    if (dev >= count) {
        set_error("sdot_server_create: no such device");
        return SDOT_ERR_ARG;
    }
    size_t budget = o.hbm_budget;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        SDOT_CUDA_TRY(cudaSetDevice(dev));
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        cudaSetDevice(cur);
        if (e != cudaSuccess) {
            set_error(std::string("sdot_server_create: cudaMemGetInfo: ") + cudaGetErrorString(e));
            return SDOT_ERR_CUDA;
        }
        budget = fr / 10 * 9;
    }
    sdot_server* srv = new sdot_server();
    srv->device = dev;
    if (o.batch_clip) srv->batcher.reset(new Batcher(dev));
    Batcher* bt = srv->batcher.get();
    srv->sched.reset(new serve::Scheduler<JobPayload>(
        budget, o.max_active, [dev, bt](JobPayload& j) { return run_job(dev, bt, j); }));
    *out = srv;
    return SDOT_OK;
}

int sdot_server_submit(sdot_server* srv, const double* pos, const double* mass, int64_t N,
                       const double box[3], const sdot_options* opt, double tol, int64_t* id) {
    set_error("");
    if (!srv || !pos || !box || !id || !(tol > 0)) {
        set_error("sdot_server_submit: need srv, pos, box, id and tol > 0");
        return SDOT_ERR_ARG;
    }
    if (!host_pointer(pos) || (mass && !host_pointer(mass))) {
        set_error("sdot_server_submit: pos and mass must be host memory");
        return SDOT_ERR_ARG;
    }
    size_t fp = 0;
    int rc = context_footprint(N, box, opt, &fp);
    if (rc) return rc;
    JobPayload p;
    p.N = N;
    for (int a = 0; a < 3; a++) p.box[a] = box[a];
    sdot_default_options(&p.opt);
    if (opt) p.opt = *opt;
    p.tol = tol;
    p.pos.assign(pos, pos + (size_t)N * 3);
    if (mass) p.mass.assign(mass, mass + (size_t)N);
    rc = srv->sched->submit(std::move(p), fp, id);
    if (rc == SDOT_ERR_OOM)
        set_error("sdot_server_submit: the job's device footprint (" + std::to_string(fp) +
                  " bytes) exceeds the server's budget");
    return rc;
}

int sdot_server_poll(sdot_server* srv, int64_t id, int* state) {
    if (!srv) return SDOT_ERR_ARG;
    return srv->sched->state(id, state);
}

int sdot_server_wait(sdot_server* srv, int64_t id, double timeout_s, int* state) {
    if (!srv) return SDOT_ERR_ARG;
    return srv->sched->wait(id, timeout_s, state);
}

int sdot_server_result(sdot_server* srv, int64_t id, double* disp, double* psi,
                       sdot_stats* st, double times[3]) {
    set_error("");
    if (!srv) return SDOT_ERR_ARG;
    JobPayload p;
    int jrc = SDOT_OK;
    double t[3] = {0, 0, 0};
    int rc = srv->sched->take(id, &p, &jrc, t);
    if (rc == SDOT_ERR_NOT_READY) {
        set_error("sdot_server_result: job " + std::to_string((long long)id) + " has not finished");
        return rc;
    }
    if (rc) {
        set_error("sdot_server_result: unknown job id");
        return rc;
    }
    if (times)
        for (int a = 0; a < 3; a++) times[a] = t[a];
    if (st) *st = p.stats;
    if (jrc != SDOT_OK) {
        set_error(p.err);
        return jrc;
    }
    if (disp) memcpy(disp, p.disp.data(), p.disp.size() * sizeof(double));
    if (psi) memcpy(psi, p.psi.data(), p.psi.size() * sizeof(double));
    return SDOT_OK;
}

int sdot_server_get_info(sdot_server* srv, sdot_server_info* info) {
    if (!srv || !info) return SDOT_ERR_ARG;
    auto f = srv->sched->info();
    info->hbm_budget = f.budget;
    info->used_bytes = f.used;
    info->peak_used_bytes = f.peak_used;
    info->max_active = f.max_active;
    info->active = f.active;
    info->peak_active = f.peak_active;
    info->queued = f.queued;
    info->finished = f.finished;
    info->submitted = f.submitted;
    return SDOT_OK;
}

void sdot_server_destroy(sdot_server* srv) {
    if (!srv) return;
    srv->sched.reset();  // waits for the running jobs, which may still use the batcher
    srv->batcher.reset();
    delete srv;
}

}  // extern "C"
