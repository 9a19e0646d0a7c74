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

#include <chrono>
#include <memory>
#include <string>
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

// one Laguerre evaluation asked for by a job's thread
struct EvalReq {
    DeviceState* d = nullptr;
    const double* psi = nullptr;
    int prec = 0;
    EvalResult* r = nullptr;
    int rc = SDOT_OK;
    std::string err;
};

// device state of the batcher's worker thread: its stream and job tables, made on
// the first batch (on that thread) and released when the thread exits
struct BatchDevice {
    int device = 0;
    bool ready = false;
    int init_rc = SDOT_OK;
    std::string init_err;
    cudaStream_t s = nullptr;
    BatchScratch* sc = nullptr;

    void init() {
        ready = true;
        if (cudaSetDevice(device) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            init_rc = SDOT_ERR_CUDA;
            init_err = std::string("batcher: ") + cudaGetErrorString(cudaGetLastError());
            return;
        }
        if ((init_rc = batch_scratch_create(MAX_BATCH, &sc)) != SDOT_OK)
            init_err = sdot_last_error();
    }

    void run(std::vector<EvalReq*>& reqs) {
        if (!ready) init();
        int rc = init_rc;
        std::string err = init_err;
        if (rc == SDOT_OK) {
            std::vector<DeviceState*> ds;
            std::vector<const double*> psis;
            std::vector<int> precs;
            std::vector<EvalResult> res(reqs.size());
            for (EvalReq* q : reqs) {
                ds.push_back(q->d);
                psis.push_back(q->psi);
                precs.push_back(q->prec);
            }
            rc = evaluate_cells_batch(ds.data(), psis.data(), precs.data(), res.data(),
                                      (int)reqs.size(), sc, s);
            if (rc == SDOT_OK)
                for (size_t t = 0; t < reqs.size(); t++) *reqs[t]->r = res[t];
            else
                err = sdot_last_error();
        }
        for (EvalReq* q : reqs) {
            q->rc = rc;
            q->err = err;
        }
    }

    void fini() {
        batch_scratch_destroy(sc);
        sc = nullptr;
        if (s) cudaStreamDestroy(s);
        s = nullptr;
    }
};

using EvalBatcher = serve::Batcher<EvalReq>;

// evaluation hook of a job's context: the job's earlier work (and psi) must be done
// before the batcher's stream reads it, and the batcher's stream is synchronised
// before the result comes back
int batched_eval(void* user, DeviceState* d, const double* psi, int prec, EvalResult* r,
                 cudaStream_t job_stream) {
    cudaError_t e = cudaStreamSynchronize(job_stream);
    if (e != cudaSuccess) {
        set_error(std::string("batched evaluation: ") + cudaGetErrorString(e));
        return SDOT_ERR_CUDA;
    }
    EvalReq q;
    q.d = d;
    q.psi = psi;
    q.prec = prec;
    q.r = r;
    static_cast<EvalBatcher*>(user)->submit(&q);
    if (q.rc != SDOT_OK) set_error(q.err);
    return q.rc;
}

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
int run_job(int device, EvalBatcher* batcher, JobPayload& j) {
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
        set_eval_hook(ctx, &batched_eval, batcher);
        batcher->add_active(1);
    }
    if (rc == SDOT_OK) rc = sdot_solve(ctx, j.tol, nullptr, &j.stats);
    if (ctx && batcher) batcher->add_active(-1);
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
    // destroyed in reverse order: the scheduler first (no job can then wait on the
    // batcher), then the batcher (its thread releases the batch device state), then
    // that state
    std::unique_ptr<BatchDevice> bdev;
    std::unique_ptr<EvalBatcher> batcher;
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
    if (o.batch_clip) {
        srv->bdev.reset(new BatchDevice());
        srv->bdev->device = dev;
        BatchDevice* bd = srv->bdev.get();
        srv->batcher.reset(new EvalBatcher(
            BATCH_WINDOW, MAX_BATCH, [bd](std::vector<EvalReq*>& reqs) { bd->run(reqs); },
            [bd] { bd->fini(); }));
    }
    EvalBatcher* bt = srv->batcher.get();
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
    srv->bdev.reset();
    delete srv;
}

}  // extern "C"
