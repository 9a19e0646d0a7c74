// C ABI of libsdot (include/sdot.h) and the host damped-Newton driver.
//
// Newton reading (the paper cites Kitagawa-Merigot-Thibert for convergence of a
// Newton method on the concave C^2 dual K, Sec. "Monge-Ampere-Kantorovich
// Reconstruction"; the damping rule is theirs): eps0 = 1/2 min(min_j V_j(psi0),
// min_j nu_j); the step is psi + alpha delta with the first alpha in 1, 1/2, 1/4 ...
// such that min_j V_j >= eps0 (no cell empties, the constraint stated beside the
// maximisation of K) and ||nu - V||_2 <= (1 - alpha/2) ||nu - V(psi)||_2.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace sdot {
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

// device allocator of new contexts (sdot_set_allocator); null: cudaMalloc / cudaFree
struct Allocator {
    void* (*alloc)(size_t, void*) = nullptr;
    void (*free)(void*, void*) = nullptr;
    void* user = nullptr;
};
static std::mutex g_alloc_mu;
static Allocator g_alloc;
}  // namespace sdot

using namespace sdot;

struct sdot_ctx {
    DeviceState d;
    sdot_options opt;
    cudaStream_t stream = 0;
    std::vector<void*> allocs;
    void* temp = nullptr;
    size_t temp_bytes = 0;
    double* stage = nullptr;  // N * 3 doubles for host <-> device staging
    int64_t nnz_cap = 0;
    int64_t nnz = 0;
    int64_t nnz_cap_u = 0;
    int64_t sell_cap = 0;     // entries the sliced-ELL arrays hold
    void* mesh_scratch = nullptr;  // sdot_mesh: fixed-point masses and phi bits
    size_t mesh_scratch_bytes = 0;
    void* mesh_stage = nullptr;    // sdot_mesh: device copies of host outputs
    size_t mesh_stage_bytes = 0;
    bool eval_valid = false;  // last evaluation is at d.psi
    float ms_knn = 0;
    EvalResult last{};
    int last_prec = SDOT_PREC_MIXED;  // precision of the last evaluation
    bool has_eval = false;            // some evaluation has run (c->last is set)
    int64_t sell_entries = 0;         // stored entries of the last Newton matrix
    int64_t sell_offdiag = 0;         // its nonzero off-diagonal entries
    bool dry = false;         // allocation plan only: count bytes, allocate nothing
    size_t bytes = 0;         // device bytes requested by the allocations so far
    EvalHook eval_hook = nullptr;  // the server's batcher, or null: evaluate_cells
    void* eval_user = nullptr;
    Allocator alloc;               // the allocator at creation (frees with the same one)
};

namespace {

int dev_alloc(sdot_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    c->bytes += (bytes + 511) / 512 * 512;
    if (c->dry) return SDOT_OK;
    if (c->alloc.alloc) {
        *p = c->alloc.alloc(bytes, c->alloc.user);
        if (!*p) {
            set_error("device allocation of " + std::to_string(bytes) +
                      " bytes failed (caller's allocator)");
            return SDOT_ERR_OOM;
        }
        c->allocs.push_back(*p);
        return SDOT_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("device allocation of ") + std::to_string(bytes) +
                  " bytes failed: " + cudaGetErrorString(e));
        return SDOT_ERR_OOM;
    }
    c->allocs.push_back(*p);
    return SDOT_OK;
}

template <typename T>
int alloc_n(sdot_ctx* c, T** p, int64_t n) {
    return dev_alloc(c, (void**)p, (size_t)n * sizeof(T));
}

void dev_free(sdot_ctx* c, void* p) {
    if (!p) return;
    for (size_t t = 0; t < c->allocs.size(); t++)
        if (c->allocs[t] == p) {
            c->allocs.erase(c->allocs.begin() + t);
            break;
        }
    if (c->alloc.free) c->alloc.free(p, c->alloc.user);
    else cudaFree(p);
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device view of a caller vector of n doubles (copies host data into dst)
int input_vec(sdot_ctx* c, const double* src, int64_t n, double* dst, const double** view) {
    if (is_device_ptr(src)) {
        *view = src;
        return SDOT_OK;
    }
    SDOT_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream));
    *view = dst;
    return SDOT_OK;
}

int check_opt(const sdot_options& o) {
    if (o.k < 1 || o.k > KMAX) return SDOT_ERR_ARG;
    if (o.precision != SDOT_PREC_FP64 && o.precision != SDOT_PREC_MIXED) return SDOT_ERR_ARG;
    if (!(o.seeds_per_leaf > 0.05 && o.seeds_per_leaf < 1000)) return SDOT_ERR_ARG;
    if (!(o.cg_rtol > 0 && o.cg_rtol < 1)) return SDOT_ERR_ARG;
    if (o.cg_maxit < 1 || o.newton_maxit < 0) return SDOT_ERR_ARG;
    if (!(o.alpha_min > 0 && o.alpha_min <= 1)) return SDOT_ERR_ARG;
    if (o.carry_certificates != 0 && o.carry_certificates != 1) return SDOT_ERR_ARG;
    return SDOT_OK;
}

int eval_at(sdot_ctx* c, const double* psi_sorted, EvalResult* r, int precision = -1) {
    const int prec = precision < 0 ? c->opt.precision : precision;
    int rc = c->eval_hook ? c->eval_hook(c->eval_user, &c->d, psi_sorted, prec, r, c->stream)
                          : evaluate_cells(c->d, psi_sorted, prec, r, c->stream);
    if (rc) return rc;
    c->last = *r;
    c->last_prec = prec;
    c->has_eval = true;
    // the context's diagram is at its current psi only for an evaluation at d.psi (a
    // line-search trial evaluates psi_trial)
    c->eval_valid = psi_sorted == c->d.psi;
    return SDOT_OK;
}

// error code for the flags of an evaluation that must be valid
int eval_status(const EvalResult& r, const char* where) {
    if (r.flags & CS_TOO_LARGE) {
        set_error(std::string(where) +
                  ": a cell reaches half a box length from its seed (too few seeds for "
                  "minimum-image distances, or psi too far from balance)");
        return SDOT_ERR_TOO_FEW;
    }
    if (r.flags & CS_CAPACITY) {
        set_error(std::string(where) + ": a cell exceeded the polytope capacity (" +
                  std::to_string(MAXP) + " planes, " + std::to_string(MAXT) + " vertices, " +
                  std::to_string(FCAP) + " facets); status bits " + std::to_string(r.flags));
        return SDOT_ERR_CAPACITY;
    }
    return SDOT_OK;
}

int ensure_csr_capacity(sdot_ctx* c, int64_t nnz) {
    if (nnz <= c->nnz_cap) return SDOT_OK;
    dev_free(c, c->d.col);
    dev_free(c, c->d.val);
    c->d.col = nullptr;
    c->d.val = nullptr;
    int64_t cap = nnz + nnz / 4 + 1024;
    int rc = alloc_n(c, &c->d.col, cap);
    if (rc) return rc;
    rc = alloc_n(c, &c->d.val, cap);
    if (rc) return rc;
    c->nnz_cap = cap;
    return SDOT_OK;
}

// assemble the sorted CSR: count (fixes nnz), grow the arrays if needed, fill
int build_csr(sdot_ctx* c) {
    NvtxRange nv("hessian_csr");
    int64_t nnz = 0;
    int rc = csr_count(c->d, &nnz, c->stream);
    if (rc) return rc;
    if ((rc = ensure_csr_capacity(c, nnz))) return rc;
    if ((rc = csr_fill(c->d, c->stream))) return rc;
    c->nnz = nnz;
    return SDOT_OK;
}

// the sliced-ELL Newton matrix: count, grow the arrays if needed, fill
int build_sell(sdot_ctx* c) {
    NvtxRange nv("newton_matrix");
    int64_t ent = 0, offd = 0;
    int rc = sell_build(c->d, &ent, &offd, c->stream);
    if (rc) return rc;
    c->sell_entries = ent;
    c->sell_offdiag = offd;
    if (ent > c->sell_cap) {
        dev_free(c, c->d.sell_col);
        dev_free(c, c->d.sell_val);
        c->d.sell_col = nullptr;
        c->d.sell_val = nullptr;
        const int64_t cap = ent + ent / 4 + 1024;
        if ((rc = alloc_n(c, &c->d.sell_col, cap))) return rc;
        if ((rc = alloc_n(c, &c->d.sell_val, cap))) return rc;
        c->sell_cap = cap;
    }
    return sell_fill(c->d, c->stream);
}

// Every device array of a context for d.N seeds in box d.L (the hash grid, kNN lists,
// facet slab, PCG vectors, psi pyramid, temp). With c->dry set nothing is allocated
// and c->bytes receives the total, which is the footprint of a server job.
int alloc_context(sdot_ctx* c) {
    DeviceState& d = c->d;
    const int64_t N = d.N;
    const double boxvol = d.L[0] * d.L[1] * d.L[2];
    int rc = SDOT_OK;
    // grid dimensions (to size the temp buffer)
    double h = cbrt(c->opt.seeds_per_leaf * boxvol / (double)N);
    int64_t ncell = 1;
    int G[3];
    for (int a = 0; a < 3; a++) {
        double g = floor(d.L[a] / h);
        if (g < 1) g = 1;
        if (g > 1024) g = 1024;
        G[a] = (int)g;
        ncell *= G[a];
    }
    if ((rc = alloc_n(c, &d.pos, N)) || (rc = alloc_n(c, &d.posf, N)) || (rc = alloc_n(c, &d.pslo, N)) || (rc = alloc_n(c, &d.ioff, N)) ||
        (rc = alloc_n(c, &d.leafc, N)) ||
        (rc = alloc_n(c, &d.perm, N)) || (rc = alloc_n(c, &d.iperm, N)) ||
        (rc = alloc_n(c, &d.nu, N)) || (rc = alloc_n(c, &d.psi, N)) ||
        (rc = alloc_n(c, &d.psi_trial, N)) || (rc = alloc_n(c, &d.knn, N * d.k)) ||
        (rc = alloc_n(c, &d.knn_d2k, N)) || (rc = alloc_n(c, &d.vol, N)) ||
        (rc = alloc_n(c, &d.m1, N * 3)) || (rc = alloc_n(c, &d.anchor, N * 3)) ||
        (rc = alloc_n(c, &d.status, N)) || (rc = alloc_n(c, &d.fcnt, N)) ||
        (rc = alloc_n(c, &d.fcol, N * FCAP)) || (rc = alloc_n(c, &d.fval, N * FCAP)) ||
        (rc = alloc_n(c, &d.topo, N * TOPO)) || (rc = alloc_n(c, &d.topo_n, N)) ||
        (rc = alloc_n(c, &d.cert_f, N * CERT_F)) || (rc = alloc_n(c, &d.cert_s, N * CERT_S)) ||
        (rc = alloc_n(c, &d.cert_j, N * CERT_NEAR)) || (rc = alloc_n(c, &d.cert_n, N)) ||
        (rc = alloc_n(c, &d.psi_prev, N)) ||
        (rc = alloc_n(c, &d.queue, N)) || (rc = alloc_n(c, &d.queue64, N)) ||
        (rc = alloc_n(c, &d.counters, 32)) || (rc = alloc_n(c, &d.row_ptr, N + 1)) ||
        (rc = alloc_n(c, &d.rowcnt, N + 1)) || (rc = alloc_n(c, &d.x, N)) ||
        (rc = alloc_n(c, &d.r, N)) || (rc = alloc_n(c, &d.z, N)) || (rc = alloc_n(c, &d.p, N)) ||
        (rc = alloc_n(c, &d.q, N)) || (rc = alloc_n(c, &d.sv, N)) || (rc = alloc_n(c, &d.uf, N)) ||
        (rc = alloc_n(c, &d.dinv, N)) || (rc = alloc_n(c, &d.sell_ptr, (N + 31) / 32 + 1)) ||
        (rc = alloc_n(c, &d.sell_w, (N + 31) / 32 + 1)) ||
        (rc = alloc_n(c, &d.partials, 1 << 20)) || (rc = alloc_n(c, &d.scal, 64)) ||
        (rc = alloc_n(c, &d.grid.cell_start, ncell + 1)) || (rc = alloc_n(c, &c->stage, N * 3)))
        return rc;
    d.delta = d.x;
    size_t tb = (size_t)(((N * 4 + 255) / 256) * 256) + 2 * (size_t)(((ncell * 4 + 255) / 256) * 256) +
                256 + scan_temp_bytes(ncell + 1) + 4096;
    if ((rc = dev_alloc(c, &c->temp, tb))) return rc;
    c->temp_bytes = tb;
    // pyramid of psi bounds: level 0 = grid cells, each level 4x coarser, top <= 4^3
    {
        Pyramid& P = d.pyr;
        int dim[3] = {G[0], G[1], G[2]};
        int64_t off = 0;
        P.nlev = 0;
        while (true) {
            for (int a = 0; a < 3; a++) P.dim[P.nlev][a] = dim[a];
            P.off[P.nlev] = off;
            off += (int64_t)dim[0] * dim[1] * dim[2];
            P.nlev++;
            if ((dim[0] <= 4 && dim[1] <= 4 && dim[2] <= 4) || P.nlev == MAXLEV) break;
            for (int a = 0; a < 3; a++) dim[a] = (dim[a] + 3) / 4;
        }
        if ((rc = alloc_n(c, &P.psimax, off))) return rc;
    }
    return SDOT_OK;
}

void log_iter(const sdot_ctx* c, int it, const EvalResult& r, double alpha, int cg_it,
              double cg_res, int trials) {
    if (!c->opt.verbose) return;
    fprintf(stderr,
            "{\"newton_it\": %d, \"max_rel_err\": %.6e, \"l2_err\": %.6e, \"min_vol\": %.6e, "
            "\"alpha\": %g, \"cg_iters\": %d, \"cg_rel_res\": %.3e, \"trials\": %d, "
            "\"requeued\": %lld, \"reclipped_fp64\": %lld, \"clip_ms\": %.3f, "
            "\"pass_ms\": [%.3f, %.3f, %.3f], \"work\": [%llu, %llu, %llu, %llu, %llu, %llu, %llu, %llu]}\n",
            it, r.max_rel_err, r.l2_err, r.min_vol, alpha, cg_it, cg_res, trials,
            (long long)r.requeued, (long long)r.reclipped, r.ms, r.ms_pass[0], r.ms_pass[1],
            r.ms_pass[2], r.work[0], r.work[1], r.work[2], r.work[3], r.work[4], r.work[5],
            r.work[6], r.work[7]);
}

}  // namespace

namespace sdot {

// sdot_create with all work on the given stream (the server creates each job's
// context on a stream of its own)
int create_context(const double* pos, const double* mass, int64_t N, const double box[3],
                   const sdot_options* opt, cudaStream_t stream, sdot_ctx** out) {
    NvtxRange nv("sdot_create");
    g_err.clear();
    if (!out) {
        set_error("sdot_create: out is NULL");
        return SDOT_ERR_ARG;
    }
    *out = nullptr;
    if (!pos || !box || N < 2 || N > (int64_t)INT32_MAX - 1) {
        set_error("sdot_create: need pos, box and 2 <= N < 2^31");
        return SDOT_ERR_ARG;
    }
    for (int a = 0; a < 3; a++)
        if (!(box[a] > 0) || !isfinite(box[a])) {
            set_error("sdot_create: box lengths must be finite and positive");
            return SDOT_ERR_ARG;
        }
    sdot_ctx* c = new sdot_ctx();
    c->stream = stream;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        c->alloc = g_alloc;
    }
    sdot_default_options(&c->opt);
    if (opt) c->opt = *opt;
    if (check_opt(c->opt)) {
        delete c;
        set_error("sdot_create: invalid options");
        return SDOT_ERR_ARG;
    }
    if (c->opt.k > N - 1) {
        delete c;
        set_error("sdot_create: k must be < N");
        return SDOT_ERR_TOO_FEW;
    }
    DeviceState& d = c->d;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.k = c->opt.k;
    d.carry = c->opt.carry_certificates;
    for (int a = 0; a < 3; a++) d.L[a] = box[a];
    const double boxvol = box[0] * box[1] * box[2];
    d.a = cbrt(boxvol / (double)N);
    int rc = SDOT_OK;
    auto fail = [&](int code) {
        sdot_destroy(c);
        return code;
    };
    if ((rc = alloc_context(c))) return fail(rc);
    cudaStream_t s = c->stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    // positions: device view (caller buffer or staging copy)
    const double* posd = nullptr;
    if ((rc = input_vec(c, pos, N * 3, c->stage, &posd))) return fail(rc);
    if ((rc = build_grid(d, posd, c->opt.seeds_per_leaf, c->temp, s, "sdot_create"))) return fail(rc);
    // masses in sorted order
    if (mass) {
        const double* md = nullptr;
        if ((rc = input_vec(c, mass, N, c->stage, &md))) return fail(rc);
        if ((rc = gather_from_user(d, md, d.nu, 1, s))) return fail(rc);
    } else {
        std::vector<double> u((size_t)N, boxvol / (double)N);
        if (cudaMemcpyAsync(d.nu, u.data(), (size_t)N * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("sdot_create: copying masses failed");
            return fail(SDOT_ERR_CUDA);
        }
    }
    {
        double msum = 0, mmin = 0;
        if ((rc = check_masses(d, &msum, &mmin, s))) return fail(rc);
        if (!(mmin > 0) || !(fabs(msum - boxvol) <= 1e-10 * boxvol)) {
            set_error("sdot_create: masses must be positive and sum to the box volume (sum " +
                      std::to_string(msum) + ", box " + std::to_string(boxvol) + ")");
            return fail(SDOT_ERR_MASS);
        }
    }
    int kflags = 0;
    if ((rc = build_knn(d, s, &kflags))) return fail(rc);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&c->ms_knn, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (kflags & 1) {
        set_error("sdot_create: two seeds share a position");
        return fail(SDOT_ERR_DUPLICATE);
    }
    if (kflags & 2) {
        set_error("sdot_create: fewer than k other seeds");
        return fail(SDOT_ERR_TOO_FEW);
    }
    if (cudaMemsetAsync(d.psi, 0, (size_t)N * 8, s) != cudaSuccess ||
        cudaMemsetAsync(d.anchor, 0, (size_t)N * 12, s) != cudaSuccess ||
        cudaMemsetAsync(d.fcnt, 0, (size_t)N * 4, s) != cudaSuccess ||
        cudaMemsetAsync(d.fcol, 0, (size_t)N * FCAP * 4, s) != cudaSuccess ||
        cudaMemsetAsync(d.fval, 0, (size_t)N * FCAP * 8, s) != cudaSuccess ||
        cudaMemsetAsync(d.topo_n, 0, (size_t)N, s) != cudaSuccess ||
        cudaMemsetAsync(d.cert_n, 0xff, (size_t)N, s) != cudaSuccess ||
        cudaMemsetAsync(d.psi_prev, 0, (size_t)N * 8, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("sdot_create: initialisation failed");
        return fail(SDOT_ERR_CUDA);
    }
    *out = c;
    return SDOT_OK;
}

void set_eval_hook(sdot_ctx* c, EvalHook hook, void* user) {
    c->eval_hook = hook;
    c->eval_user = user;
}

// device bytes of a context for N seeds (the allocations of create_context, counted
// without allocating) plus a reserve for the CSR Hessian of sdot_solve
int context_footprint(int64_t N, const double box[3], const sdot_options* opt, size_t* bytes) {
    if (!bytes || !box || N < 2 || N > (int64_t)INT32_MAX - 1) {
        set_error("sdot_server_footprint: need box, bytes and 2 <= N < 2^31");
        return SDOT_ERR_ARG;
    }
    for (int a = 0; a < 3; a++)
        if (!(box[a] > 0) || !isfinite(box[a])) {
            set_error("sdot_server_footprint: box lengths must be finite and positive");
            return SDOT_ERR_ARG;
        }
    sdot_ctx c;
    c.dry = true;
    sdot_default_options(&c.opt);
    if (opt) c.opt = *opt;
    if (check_opt(c.opt) || c.opt.k > N - 1) {
        set_error("sdot_server_footprint: invalid options (or k >= N)");
        return SDOT_ERR_ARG;
    }
    DeviceState& d = c.d;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.k = c.opt.k;
    for (int a = 0; a < 3; a++) d.L[a] = box[a];
    d.a = cbrt(box[0] * box[1] * box[2] / (double)N);
    int rc = alloc_context(&c);
    if (rc) return rc;
    // Newton matrix: 25 entries per seed (int32 column + 8-byte value), the sliced-ELL
    // capacity sdot_solve grows to on Zel'dovich boxes (about 17 entries per row padded
    // to the longest row of each slice of 32, 25% headroom)
    *bytes = c.bytes + ((size_t)N * 25 * 12 + 511) / 512 * 512;
    return SDOT_OK;
}

}  // namespace sdot

extern "C" {

const char* sdot_last_error(void) { return g_err.c_str(); }

int64_t sdot_kernel_launches(void) { return (int64_t)launch_count(); }

int sdot_default_options(sdot_options* o) {
    if (!o) return SDOT_ERR_ARG;
    o->k = 24;
    o->precision = SDOT_PREC_MIXED;
    o->seeds_per_leaf = 2.0;
    o->cg_rtol = 1e-3;
    o->cg_maxit = 5000;
    o->newton_maxit = 100;
    o->alpha_min = 1.0 / (1 << 30);
    o->verbose = 0;
    o->warm_alpha = 1;
    o->carry_certificates = 1;
    return SDOT_OK;
}

void sdot_destroy(sdot_ctx* c) {
    if (!c) return;
    for (void* p : c->allocs) {
        if (c->alloc.free) c->alloc.free(p, c->alloc.user);
        else cudaFree(p);
    }
    c->allocs.clear();
    delete c;
}

int sdot_set_allocator(void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*), void* user) {
    g_err.clear();
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("sdot_set_allocator: give both alloc and free, or neither");
        return SDOT_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free = free_fn;
    g_alloc.user = alloc ? user : nullptr;
    return SDOT_OK;
}

int sdot_set_stream(sdot_ctx* c, void* stream) {
    if (!c) return SDOT_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return SDOT_OK;
}

int sdot_mesh(sdot_ctx* c, double lambda, int mesh, double* rho, double* phi, int32_t* owner) {
    g_err.clear();
    if (!c || mesh < 1 || mesh > 2048 || !(lambda >= 0.0 && lambda < 1.0) ||
        (!rho && !phi && !owner)) {
        set_error("sdot_mesh: need a context, 1 <= mesh <= 2048, 0 <= lambda < 1 and an output");
        return SDOT_ERR_ARG;
    }
    DeviceState& d = c->d;
    cudaStream_t s = c->stream;
    int rc;
    if (!c->eval_valid) {
        EvalResult r;
        if ((rc = eval_at(c, d.psi, &r))) return rc;
        if ((rc = eval_status(r, "sdot_mesh"))) return rc;
    }
    const int64_t n = (int64_t)mesh * mesh * mesh;
    auto grow = [&](void** p, size_t* have, size_t need) -> int {
        if (need <= *have) return SDOT_OK;
        dev_free(c, *p);
        *p = nullptr;
        *have = 0;
        int r = dev_alloc(c, p, need);
        if (r) return r;
        *have = need;
        return SDOT_OK;
    };
    if ((rc = grow(&c->mesh_scratch, &c->mesh_scratch_bytes, (size_t)n * 16))) return rc;
    const bool rho_dev = !rho || is_device_ptr(rho), phi_dev = !phi || is_device_ptr(phi),
               own_dev = !owner || is_device_ptr(owner);
    const size_t stage = (rho_dev ? 0 : 8) + (phi_dev ? 0 : 8) + (own_dev ? 0 : 4);
    if (stage && (rc = grow(&c->mesh_stage, &c->mesh_stage_bytes, (size_t)n * stage))) return rc;
    char* sp = (char*)c->mesh_stage;
    double* rho_d = rho_dev ? rho : (double*)sp;
    if (!rho_dev) sp += (size_t)n * 8;
    double* phi_d = phi_dev ? phi : (double*)sp;
    if (!phi_dev) sp += (size_t)n * 8;
    int32_t* own_d = own_dev ? owner : (int32_t*)sp;
    if ((rc = mesh_eval(d, mesh, lambda, rho_d, phi_d, own_d, c->mesh_scratch, s))) return rc;
    if (!rho_dev) SDOT_CUDA_TRY(cudaMemcpyAsync(rho, rho_d, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    if (!phi_dev) SDOT_CUDA_TRY(cudaMemcpyAsync(phi, phi_d, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    if (!own_dev) SDOT_CUDA_TRY(cudaMemcpyAsync(owner, own_d, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    return SDOT_OK;
}

int sdot_last_eval(const sdot_ctx* c, sdot_eval_info* info) {
    if (!c || !info) {
        set_error("sdot_last_eval: need a context and info");
        return SDOT_ERR_ARG;
    }
    if (!c->has_eval) {
        set_error("sdot_last_eval: the context has not been evaluated yet");
        return SDOT_ERR_ARG;
    }
    const EvalResult& r = c->last;
    info->ms_clip = r.ms;
    for (int q = 0; q < 3; q++) info->ms_pass[q] = r.ms_pass[q];
    info->requeued = r.requeued;
    info->reclipped_fp64 = r.reclipped;
    info->n_empty = r.n_empty;
    info->max_rel_err = r.max_rel_err;
    info->l2_err = r.l2_err;
    info->min_vol = r.min_vol;
    info->precision = c->last_prec;
    info->carried = r.carried;
    return SDOT_OK;
}

int sdot_size(const sdot_ctx* c, int64_t* N, int* k) {
    if (!c) return SDOT_ERR_ARG;
    if (N) *N = c->d.N;
    if (k) *k = c->d.k;
    return SDOT_OK;
}

int sdot_create(const double* pos, const double* mass, int64_t N, const double box[3],
                const sdot_options* opt, sdot_ctx** out) {
    return create_context(pos, mass, N, box, opt, 0, out);
}

int sdot_laguerre(sdot_ctx* c, const double* psi, double* volumes, double* centroids,
                  sdot_csr* hess) {
    NvtxRange nv("sdot_laguerre");
    g_err.clear();
    if (!c) return SDOT_ERR_ARG;
    DeviceState& d = c->d;
    cudaStream_t s = c->stream;
    int rc;
    if (psi) {
        const double* pv = nullptr;
        if ((rc = input_vec(c, psi, d.N, c->stage, &pv))) return rc;
        // checked in the scratch vector first: a rejected psi leaves the context as it was
        if ((rc = gather_from_user(d, pv, d.psi_trial, 1, s))) return rc;
        bool ok = false;
        if ((rc = all_finite(d, d.psi_trial, d.N, &ok, s))) return rc;
        if (!ok) {
            set_error("sdot_laguerre: psi has a non-finite entry");
            return SDOT_ERR_ARG;
        }
        SDOT_CUDA_TRY(cudaMemcpyAsync(d.psi, d.psi_trial, (size_t)d.N * 8,
                                      cudaMemcpyDeviceToDevice, s));
    }
    EvalResult r;
    if ((rc = eval_at(c, d.psi, &r))) return rc;
    c->last = r;
    c->eval_valid = true;
    if ((rc = eval_status(r, "sdot_laguerre"))) return rc;
    auto out_vec = [&](double* dst, int w, bool cen) -> int {
        bool dev = is_device_ptr(dst);
        double* tgt = dev ? dst : c->stage;
        int q = cen ? centroids_user(d, tgt, 1, s) : scatter_to_user(d, d.vol, tgt, w, s);
        if (q) return q;
        if (!dev) {
            SDOT_CUDA_TRY(cudaMemcpyAsync(dst, tgt, (size_t)d.N * w * 8, cudaMemcpyDeviceToHost, s));
            SDOT_CUDA_TRY(cudaStreamSynchronize(s));
        }
        return SDOT_OK;
    };
    if (volumes && (rc = out_vec(volumes, 1, false))) return rc;
    if (centroids && (rc = out_vec(centroids, 3, true))) return rc;
    if (hess) {
        if ((rc = build_csr(c))) return rc;
        if (c->nnz > c->nnz_cap_u) {
            dev_free(c, d.col_u);
            dev_free(c, d.val_u);
            d.col_u = nullptr;
            d.val_u = nullptr;
            if (!d.row_ptr_u && (rc = alloc_n(c, &d.row_ptr_u, d.N + 1))) return rc;
            if ((rc = alloc_n(c, &d.col_u, c->nnz_cap)) || (rc = alloc_n(c, &d.val_u, c->nnz_cap)))
                return rc;
            c->nnz_cap_u = c->nnz_cap;
        }
        if ((rc = assemble_csr_user(d, c->nnz, s))) return rc;
        SDOT_CUDA_TRY(cudaStreamSynchronize(s));
        hess->n = d.N;
        hess->nnz = c->nnz;
        hess->row_ptr = d.row_ptr_u;
        hess->col = d.col_u;
        hess->val = d.val_u;
    }
    if (r.n_empty > 0) {
        set_error("sdot_laguerre: " + std::to_string(r.n_empty) + " empty cell(s)");
        return SDOT_ERR_EMPTY_CELL;
    }
    return SDOT_OK;
}

int sdot_solve(sdot_ctx* c, double tol, const double* psi0, sdot_stats* st) {
    NvtxRange nv("sdot_solve");
    g_err.clear();
    if (!c || !(tol > 0)) {
        set_error("sdot_solve: need a context and tol > 0");
        return SDOT_ERR_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    DeviceState& d = c->d;
    cudaStream_t s = c->stream;
    int rc;
    sdot_stats S;
    memset(&S, 0, sizeof S);
    S.ms_knn = c->ms_knn;
    if (psi0) {
        const double* pv = nullptr;
        if ((rc = input_vec(c, psi0, d.N, c->stage, &pv))) return rc;
        // checked in the scratch vector first: a rejected psi0 leaves the context as it was
        if ((rc = gather_from_user(d, pv, d.psi_trial, 1, s))) return rc;
        bool ok = false;
        if ((rc = all_finite(d, d.psi_trial, d.N, &ok, s))) return rc;
        if (!ok) {
            set_error("sdot_solve: psi0 has a non-finite entry");
            return SDOT_ERR_ARG;
        }
        SDOT_CUDA_TRY(cudaMemcpyAsync(d.psi, d.psi_trial, (size_t)d.N * 8,
                                      cudaMemcpyDeviceToDevice, s));
    } else {
        SDOT_CUDA_TRY(cudaMemsetAsync(d.psi, 0, (size_t)d.N * 8, s));
    }
    if ((rc = subtract_mean(d, d.psi, s))) return rc;
    EvalResult ev;
    if ((rc = eval_at(c, d.psi, &ev))) return rc;
    c->eval_valid = true;
    S.laguerre_evals = 1;
    S.ms_clip += ev.ms;
    for (int q = 0; q < 3; q++) S.ms_pass[q] += ev.ms_pass[q];
    if (c->opt.precision == SDOT_PREC_MIXED) {
        S.evals_fp32++;
        S.ms_pass1_fp32 += ev.ms_pass[0];
    }
    if ((rc = eval_status(ev, "sdot_solve"))) return rc;
    if (ev.n_empty > 0) {
        set_error("sdot_solve: the initial psi has empty cells");
        return SDOT_ERR_EMPTY_CELL;
    }
    double numin = 0, nusum = 0;
    if ((rc = check_masses(d, &nusum, &numin, s))) return rc;
    const double eps0 = 0.5 * fmin(ev.min_vol, numin);
    cudaEvent_t c0, c1;
    cudaEventCreate(&c0);
    cudaEventCreate(&c1);
    int it = 0;
    double alpha = 1.0;
    int prec = c->opt.precision;  // precision of the current evaluations
    rc = SDOT_OK;
    log_iter(c, it, ev, 0.0, 0, 0.0, 0);
    while (!(ev.max_rel_err <= tol)) {
        if (!std::isfinite(ev.max_rel_err)) {
            set_error("sdot_solve: non-finite cell volumes (psi far outside the range of "
                      "the box geometry)");
            rc = SDOT_ERR_ARG;
            break;
        }
        if (it >= c->opt.newton_maxit) {
            set_error("sdot_solve: Newton reached newton_maxit");
            rc = SDOT_ERR_MAXIT;
            break;
        }
        if ((rc = build_sell(c))) break;
        int cg_it = 0;
        double cg_res = 0;
        cudaEventRecord(c0, s);
        if ((rc = cg_solve(d, c->opt.cg_rtol, c->opt.cg_maxit, &cg_it, &cg_res, s))) break;
        cudaEventRecord(c1, s);
        cudaEventSynchronize(c1);
        float ms = 0;
        cudaEventElapsedTime(&ms, c0, c1);
        S.ms_cg += ms;
        S.cg_iters += cg_it;
        // damping: alpha = 1, 1/2, 1/4, ... (first acceptable); with warm_alpha the
        // sequence starts at min(1, 4 alpha_prev) instead of 1
        alpha = (c->opt.warm_alpha && it > 0) ? fmin(1.0, 4.0 * alpha) : 1.0;
        int trials = 0;
        bool refine = false;
        EvalResult et;
        while (true) {
            if ((rc = axpy_gauge(d, d.psi, d.x, alpha, d.psi_trial, s))) break;
            if ((rc = eval_at(c, d.psi_trial, &et, prec))) break;
            trials++;
            S.laguerre_evals++;
            S.ms_clip += et.ms;
            for (int q = 0; q < 3; q++) S.ms_pass[q] += et.ms_pass[q];
            if (prec == SDOT_PREC_MIXED) {
                S.evals_fp32++;
                S.ms_pass1_fp32 += et.ms_pass[0];
            }
            bool valid = !(et.flags & (CS_TOO_LARGE | CS_CAPACITY));
            if (c->opt.verbose > 1)
                fprintf(stderr,
                        "{\"trial_alpha\": %g, \"flags\": %u, \"min_vol\": %.6e, \"l2_err\": %.6e, "
                        "\"target\": %.6e, \"sum_vol_rel\": %.3e, \"requeued\": %lld, \"reclipped\": %lld}\n",
                        alpha, et.flags, et.min_vol, et.l2_err, (1.0 - 0.5 * alpha) * ev.l2_err,
                        et.sum_vol / (d.L[0] * d.L[1] * d.L[2]) - 1.0, (long long)et.requeued,
                        (long long)et.reclipped);
            if (valid && et.min_vol >= eps0 && et.l2_err <= (1.0 - 0.5 * alpha) * ev.l2_err) break;
            alpha *= 0.5;
            // FP64 refinement: in the quadratic regime (small error) the full Newton
            // step must be accepted; if the FP32 cells cannot make the residual drop,
            // their rounding is the floor: the current point is evaluated again with
            // FP64 cells and the remaining Newton steps stay in FP64
            if (prec == SDOT_PREC_MIXED && ev.max_rel_err < 1e-3 && alpha < 1.0) {
                refine = true;
                break;
            }
            if (alpha < c->opt.alpha_min) {
                set_error("sdot_solve: line search step below alpha_min");
                rc = SDOT_ERR_NO_DESCENT;
                break;
            }
        }
        if (rc) break;
        if (refine) {
            prec = SDOT_PREC_FP64;
            S.refined_fp64 = 1;
            if ((rc = eval_at(c, d.psi, &ev, prec))) break;
            S.laguerre_evals++;
            S.ms_clip += ev.ms;
            for (int q = 0; q < 3; q++) S.ms_pass[q] += ev.ms_pass[q];
            alpha = 1.0;
            log_iter(c, it, ev, 0.0, cg_it, cg_res, trials);
            continue;
        }
        double* t = d.psi;
        d.psi = d.psi_trial;
        d.psi_trial = t;
        if ((rc = subtract_mean(d, d.psi, s))) break;
        ev = et;
        it++;
        log_iter(c, it, ev, alpha, cg_it, cg_res, trials);
    }
    cudaEventDestroy(c0);
    cudaEventDestroy(c1);
    c->last = ev;
    c->eval_valid = true;
    S.newton_iters = it;
    S.hess_slots = c->sell_entries;
    S.hess_offdiag = c->sell_offdiag;
    S.max_rel_err = ev.max_rel_err;
    S.l2_err = ev.l2_err;
    S.min_vol = ev.min_vol;
    S.last_alpha = alpha;
    S.requeued = ev.requeued;
    S.reclipped_fp64 = ev.reclipped;
    cudaStreamSynchronize(s);
    S.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (st) *st = S;
    return rc;
}

int sdot_csr_copy(const sdot_csr* h, int64_t* row_ptr, int32_t* col, double* val) {
    g_err.clear();
    if (!h || !row_ptr || !col || !val) {
        set_error("sdot_csr_copy: NULL argument");
        return SDOT_ERR_ARG;
    }
    SDOT_CUDA_TRY(cudaMemcpy(row_ptr, h->row_ptr, (size_t)(h->n + 1) * 8, cudaMemcpyDefault));
    SDOT_CUDA_TRY(cudaMemcpy(col, h->col, (size_t)h->nnz * 4, cudaMemcpyDefault));
    SDOT_CUDA_TRY(cudaMemcpy(val, h->val, (size_t)h->nnz * 8, cudaMemcpyDefault));
    return SDOT_OK;
}

int sdot_get_psi(sdot_ctx* c, double* psi) {
    g_err.clear();
    if (!c || !psi) return SDOT_ERR_ARG;
    DeviceState& d = c->d;
    bool dev = is_device_ptr(psi);
    double* tgt = dev ? psi : c->stage;
    int rc = scatter_to_user(d, d.psi, tgt, 1, c->stream);
    if (rc) return rc;
    if (!dev) SDOT_CUDA_TRY(cudaMemcpyAsync(psi, tgt, (size_t)d.N * 8, cudaMemcpyDeviceToHost, c->stream));
    SDOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SDOT_OK;
}

int sdot_displacement(sdot_ctx* c, double* disp) {
    g_err.clear();
    if (!c || !disp) return SDOT_ERR_ARG;
    DeviceState& d = c->d;
    int rc;
    if (!c->eval_valid) {
        EvalResult r;
        if ((rc = eval_at(c, d.psi, &r))) return rc;
        c->last = r;
        c->eval_valid = true;
        if ((rc = eval_status(r, "sdot_displacement"))) return rc;
    }
    bool dev = is_device_ptr(disp);
    double* tgt = dev ? disp : c->stage;
    if ((rc = centroids_user(d, tgt, 0, c->stream))) return rc;
    if (!dev)
        SDOT_CUDA_TRY(cudaMemcpyAsync(disp, tgt, (size_t)d.N * 24, cudaMemcpyDeviceToHost, c->stream));
    SDOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SDOT_OK;
}

int sdot_cell_status(sdot_ctx* c, uint8_t* status) {
    g_err.clear();
    if (!c || !status) return SDOT_ERR_ARG;
    DeviceState& d = c->d;
    bool dev = is_device_ptr(status);
    uint8_t* tgt = status;
    int rc;
    if (!dev && (rc = alloc_n(c, &tgt, d.N))) return rc;
    rc = status_to_user(d, tgt, c->stream);
    if (!rc && !dev &&
        cudaMemcpyAsync(status, tgt, (size_t)d.N, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        rc = SDOT_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = SDOT_ERR_CUDA;
    if (!dev) dev_free(c, tgt);
    if (rc == SDOT_ERR_CUDA) set_error("sdot_cell_status: copy failed");
    return rc;
}

int sdot_knn(sdot_ctx* c, int32_t* nbr) {
    g_err.clear();
    if (!c || !nbr) return SDOT_ERR_ARG;
    DeviceState& d = c->d;
    bool dev = is_device_ptr(nbr);
    int32_t* tgt = nbr;
    int rc;
    if (!dev && (rc = alloc_n(c, &tgt, d.N * d.k))) return rc;
    rc = knn_to_user(d, tgt, c->stream);
    if (!rc && !dev &&
        cudaMemcpyAsync(nbr, tgt, (size_t)d.N * d.k * 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        rc = SDOT_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = SDOT_ERR_CUDA;
    if (!dev) dev_free(c, tgt);
    if (rc == SDOT_ERR_CUDA) set_error("sdot_knn: copy failed");
    return rc;
}

}  // extern "C"
