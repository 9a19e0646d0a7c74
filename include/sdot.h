/*
 * sdot.h — semi-discrete optimal transport on one GPU (sm_103a), C ABI.
 *
 * Problem (arXiv:2110.08868, Sec. "Monge-Ampere-Kantorovich Reconstruction"):
 * N points y_j with masses nu_j sit in a periodic box of volume |B| = sum_j nu_j
 * (uniform Lagrangian density rho_I = 1). The library finds the weights psi_j that
 * maximise the semi-discrete Kantorovich dual, eq. (SDK),
 *     K(psi) = sum_j int_{V_j} [1/2 |y_j - q|^2 - psi_j] dq + sum_j nu_j psi_j,
 * whose Laguerre cells, eq. (laguerrecell),
 *     V_j = { q : 1/2|y_j - q|^2 - psi_j < 1/2|y_k - q|^2 - psi_k  for all k != j },
 * then all have volume nu_j. Distances are periodic (minimum image).
 *
 * Conventions for every call:
 *  - Return value: SDOT_OK (0) or a negative SDOT_ERR_* code; sdot_last_error()
 *    then gives a message (per calling thread).
 *  - Vector arguments are plain pointers to host OR device memory; the library
 *    inspects each pointer (cudaPointerGetAttributes) and copies as needed. The
 *    caller owns every buffer it passes; nothing is retained after the call
 *    returns, except where stated (borrowed CSR pointers).
 *  - All index spaces are the caller's order 0..N-1.
 *  - Work is issued on the context's stream (default: the legacy default stream;
 *    see sdot_set_stream). Calls that return host data synchronise that stream.
 *  - A context is not thread-safe; different contexts are independent.
 */
#ifndef SDOT_H
#define SDOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SDOT_OK = 0,
    SDOT_ERR_ARG = -1,        /* invalid argument (NULL, N < 2, bad option, non-finite input) */
    SDOT_ERR_MASS = -2,       /* |sum nu - |box|| > 1e-10 |box| or a mass <= 0 */
    SDOT_ERR_DUPLICATE = -3,  /* two seeds at the same position */
    SDOT_ERR_TOO_FEW = -4,    /* a cell reaches half a box: too few seeds for minimum image */
    SDOT_ERR_OOM = -5,        /* device allocation failed */
    SDOT_ERR_NO_DESCENT = -6, /* line search step fell below alpha_min */
    SDOT_ERR_MAXIT = -7,      /* Newton did not reach tol within newton_maxit */
    SDOT_ERR_EMPTY_CELL = -8, /* a Laguerre cell is empty at the given psi */
    SDOT_ERR_TIMEOUT = -9,    /* a bounded device wait gave up */
    SDOT_ERR_CUDA = -10,      /* CUDA runtime error */
    SDOT_ERR_CAPACITY = -11,  /* a cell exceeded the fixed polytope capacity even in FP64 */
    SDOT_ERR_NOT_READY = -12  /* a server job has not finished yet */
};

enum {
    SDOT_PREC_FP64 = 0,  /* clipping in FP64 */
    SDOT_PREC_MIXED = 1  /* clipping in FP32 in a frame at each cell's previous centroid,
                            FP64 plane offsets and accumulation, FP64 re-clip of cells
                            failing the consistency check */
};

typedef struct {
    int k;                 /* neighbours per seed in the kNN list (1..64, default 24) */
    int precision;         /* SDOT_PREC_FP64 or SDOT_PREC_MIXED (default MIXED) */
    double seeds_per_leaf; /* mean seeds per grid cell of the spatial hash (default 2) */
    double cg_rtol;        /* PCG stop: ||r|| <= cg_rtol ||g|| (default 1e-3) */
    int cg_maxit;          /* PCG iteration cap per Newton step (default 5000) */
    int newton_maxit;      /* Newton iteration cap (default 100) */
    double alpha_min;      /* smallest damping step before SDOT_ERR_NO_DESCENT (2^-30) */
    int verbose;           /* 1: one JSON line per Newton iteration on stderr */
    int warm_alpha;        /* 1 (default): each line search starts at min(1, 4 alpha_prev)
                              instead of 1; 0: always 1, 1/2, 1/4, ... */
    int carry_certificates; /* 1 (default): a cell's security walk is replaced by the
                              certificate of its previous walk while that still holds
                              (psi_j - psi_i moved by less than 0.01 a^2 and the cell by
                              less than 0.01 a; the seeds within those reserves are
                              re-tested exactly); 0: every evaluation walks every cell */
} sdot_options;

/* The Hessian in CSR form. L = -Hessian(K) is the weighted graph Laplacian
 * L_ij = -A_ij / |d_ij| (A_ij: facet area, d_ij: min-image seed difference),
 * L_ii = -sum_{j != i} L_ij. Device pointers, owned by the context, valid until the
 * next sdot_laguerre / sdot_solve / sdot_destroy on it. Row i holds the diagonal
 * first, then the off-diagonal entries in increasing column order. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t* row_ptr; /* n + 1 */
    const int32_t* col;     /* nnz */
    const double* val;      /* nnz */
} sdot_csr;

typedef struct {
    int newton_iters;
    int laguerre_evals;      /* cell-diagram evaluations, line-search trials included */
    int64_t cg_iters;        /* total PCG iterations */
    double max_rel_err;      /* max_j |V_j - nu_j| / nu_j at return */
    double l2_err;           /* ||V - nu||_2 at return */
    double min_vol;          /* min_j V_j at return */
    double last_alpha;       /* damping factor of the last step */
    int64_t requeued;        /* cells re-queued by the security test (last evaluation) */
    int64_t reclipped_fp64;  /* cells re-clipped in FP64 (last evaluation) */
    double ms_knn;           /* device time of the kNN build (sdot_create) */
    double ms_clip;          /* device time in cell clipping (all evaluations) */
    double ms_cg;            /* device time in PCG */
    double ms_total;         /* wall time of the solve */
    double ms_pass[3];       /* device time per clipping pass, summed over evaluations:
                                security-test pass, re-queue pass, FP64 re-clip pass */
    int refined_fp64;        /* 1 if a mixed-precision solve finished with FP64 evaluations */
    int evals_fp32;          /* evaluations with FP32 clipping */
    double ms_pass1_fp32;    /* device time of their first (security-test) pass */
    int64_t hess_slots;      /* stored entries of the last Newton matrix (sliced-ELL:
                                each slice of 32 rows padded to its longest row) */
    int64_t hess_offdiag;    /* its nonzero off-diagonal entries */
} sdot_stats;

/* The last Laguerre evaluation of a context (sdot_laguerre or the last one of
 * sdot_solve). */
typedef struct {
    double ms_clip;          /* device time of the clipping passes */
    double ms_pass[3];       /* security-test pass, re-queue pass, FP64 re-clip pass */
    int64_t requeued;        /* cells re-queued by the security test */
    int64_t reclipped_fp64;  /* cells re-clipped in FP64 */
    int64_t n_empty;         /* empty cells */
    double max_rel_err;      /* max_j |V_j - nu_j| / nu_j */
    double l2_err;           /* ||V - nu||_2 */
    double min_vol;          /* min_j V_j */
    int precision;           /* SDOT_PREC_* of the clipping */
    int64_t carried;         /* cells whose security walk a carried certificate replaced:
                                the previous evaluation's walk, with reserves of 0.01 a in
                                the cell's bounds and 0.01 a^2 in the change of psi_j -
                                psi_i, plus an exact re-test of the seeds within them */
} sdot_eval_info;

typedef struct sdot_ctx sdot_ctx;

/* Fill *opt with the defaults listed in sdot_options. */
int sdot_default_options(sdot_options* opt);

/*
 * Create a context for N seeds and build the grid hash and the kNN lists.
 *  pos:  N x 3 doubles, row-major (x, y, z); every coordinate in [0, box[a]).
 *  mass: N doubles, each > 0, summing to box[0]*box[1]*box[2] within 1e-10
 *        relative (eq. SDK with rho_I = 1); NULL means uniform |box| / N.
 *  box:  3 box lengths (host memory).
 *  opt:  NULL for defaults. Copied.
 * The seeds are sorted internally by grid cell; results are returned in the
 * caller's order. On error *out is NULL.
 */
int sdot_create(const double* pos, const double* mass, int64_t N, const double box[3],
                const sdot_options* opt, sdot_ctx** out);

/* Issue all later work of ctx on this cudaStream_t (NULL: legacy default stream). */
int sdot_set_stream(sdot_ctx* ctx, void* stream);

/*
 * Device allocator for the contexts created after this call (process-wide; both NULL
 * restores cudaMalloc / cudaFree). alloc(bytes, user) returns device memory aligned to
 * at least 256 bytes, or NULL, in which case the call that needed it fails with
 * SDOT_ERR_OOM; free(ptr, user) releases a pointer alloc returned. A context keeps
 * the allocator it was created with and frees through it. Give both functions or
 * neither (else SDOT_ERR_ARG). The library's other device memory (the server's batch
 * tables, the fixed array of sdot_knn_static) does not go through the allocator.
 */
int sdot_set_allocator(void* (*alloc)(size_t bytes, void* user),
                       void (*free)(void* ptr, void* user), void* user);

/*
 * One evaluation of the Laguerre diagram at psi (eq. laguerrecell) with the
 * quantities of eq. (SDK) and its derivatives.
 *  psi:       N doubles, or NULL for the context's current psi (0 after create).
 *             A non-NULL psi also becomes the current psi.
 *  volumes:   N doubles out (|V_j|) or NULL.
 *  centroids: N x 3 doubles out (absolute, wrapped into the box) or NULL.
 *  hess:      out, L = -Hessian(K) in the caller's index order, or NULL.
 * Returns SDOT_ERR_EMPTY_CELL (outputs still written) if some cell is empty, and
 * SDOT_ERR_ARG (context unchanged) if psi has a non-finite entry.
 */
int sdot_laguerre(sdot_ctx* ctx, const double* psi, double* volumes, double* centroids,
                  sdot_csr* hess);

/*
 * Damped Newton maximisation of K (concave and C^2, Sec. "Monge-Ampere-Kantorovich
 * Reconstruction") from psi0 (N doubles; NULL: 0) until
 * max_j |V_j - nu_j| / nu_j <= tol. Each step solves L delta = nu - V by
 * Jacobi-preconditioned CG to opt.cg_rtol (L in sliced-ELL form with FP32 weights and
 * FP32 arithmetic per stored entry, vectors and dot products in FP64: the direction is
 * an inexact solve, and the precision of the answer is that of the evaluations, which
 * decide every step) and takes the first alpha in a0, a0/2, a0/4, ... with
 * min_j V_j >= eps0 and ||nu - V||_2 <= (1 - alpha/2) ||nu - V(psi)||_2, where
 * eps0 = 1/2 min(min_j V_j(psi0), min_j nu_j); a0 = 1, or min(1, 4 alpha_prev) after
 * the first step when opt.warm_alpha is set. In mixed precision, when the error is
 * below 1e-3 and the full step alpha = 1 is rejected (FP32 rounding is the floor),
 * the current point is evaluated again with FP64 cells and the remaining Newton steps
 * stay FP64 (st->refined_fp64 = 1). The result keeps sum(psi) = 0.
 * A psi0 with a non-finite entry is refused (SDOT_ERR_ARG) and leaves the context as
 * it was. st may be NULL.
 */
int sdot_solve(sdot_ctx* ctx, double tol, const double* psi0, sdot_stats* st);

/* Copy a CSR returned by sdot_laguerre into caller buffers (host or device):
 * row_ptr n + 1 int64, col nnz int32, val nnz doubles. */
int sdot_csr_copy(const sdot_csr* h, int64_t* row_ptr, int32_t* col, double* val);

/* Current psi (N doubles out, sum zero after a solve). */
int sdot_get_psi(sdot_ctx* ctx, double* psi);

/*
 * Displacement of every cell at the current psi: disp_j = y_j - centroid(V_j),
 * minimum image (N x 3 doubles out). Each cell is mapped to its point (last
 * paragraph of Sec. "Monge-Ampere-Kantorovich Reconstruction"); this is the
 * Zel'dovich displacement of that mass element.
 */
int sdot_displacement(sdot_ctx* ctx, double* disp);

/* The kNN lists built by sdot_create: N x k int32 out, neighbours of seed j in
 * increasing (min-image d^2, index) order, d^2 = (dx*dx + dy*dy) + dz*dz in IEEE
 * binary64 without fused multiply-add. */
int sdot_knn(sdot_ctx* ctx, int32_t* nbr);

/* Per-cell status of the last evaluation (N bytes out, caller order). Bits:
 * 1 empty, 2 capacity exceeded, 4 failed the FP32 consistency check (then
 * re-clipped in FP64), 8 re-queued by the security test, 16 reaches a non-minimum
 * periodic image, 32/64/128 capacity detail (polytope / face / traversal stack).
 * A cell that went through the re-queue pass keeps bit 8, and a cell re-clipped in FP64
 * with the large polytope keeps the bits that sent it there (4, or 32/64/128 when the
 * small polytope overflowed); 1, 2 and 16 describe the final result. */
int sdot_cell_status(sdot_ctx* ctx, uint8_t* status);

/*
 * sdot_knn_static — the kNN lists of sdot_create/sdot_knn computed without allocating
 * any device memory (the paper has no counterpart; this serves callers that cannot
 * allocate on their path, e.g. code running inside another framework's memory pool or
 * under a fixed device-memory budget, or latency-critical code that must not call
 * cudaMalloc/cudaFree because they can synchronise the device).
 *  pos:    N x 3 doubles in device (or managed) memory, each coordinate in [0, box[a]).
 *  N, k:   2 <= N <= SDOT_STATIC_MAX_N, 1 <= k <= SDOT_STATIC_MAX_K, k < N; larger
 *          requests return SDOT_ERR_ARG with a message.
 *  box:    3 box lengths (host memory).
 *  nbr:    N x k int32 out, device (or managed) memory; same contents as sdot_knn.
 *  stream: cudaStream_t for the work (NULL: legacy default stream); the call returns
 *          after synchronising it.
 * All scratch lives in one fixed array of about 7 MB declared in the library, which
 * every GPU that loads the library keeps until the process exits. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture. Calls share the array and it keeps the last
 * call's contents: calls whose GPU work overlaps race, so serialise them.
 */
#define SDOT_STATIC_MAX_N 32768
#define SDOT_STATIC_MAX_K 32
int sdot_knn_static(const double* pos, int64_t N, const double box[3], int k, int32_t* nbr,
                    void* stream);

/*
 * Power spectrum of a density mesh: the estimator of the fractional BAO signal
 * d(k) = P_wig(k) / P_nw(k) - 1 that compares the densities reconstructed (sdot_mesh)
 * from a wiggle / no-wiggle pair (Sec. "BAO reconstruction", Fig. 2).
 *  rho:    M^3 doubles (host or device), indexed (z M + y) M + x like sdot_mesh's, of a
 *          periodic cubic box of side L; its mean must be positive.
 *  M:      2 ... 1024.   L: the box side (> 0).
 *  nbins:  1 ... 2 M bins; bin b = 1 ... nbins holds the modes k = 2 pi n / L with
 *          b - 1/2 <= |n| < b + 1/2 (n integer, every mode of the full transform once).
 *  P:      nbins doubles out (host): the mean over the bin's modes of L^3 |delta_k|^2,
 *          delta = rho / mean(rho) - 1, delta_k its discrete transform divided by M^3.
 *  kmean:  nbins doubles out (host) or NULL: the mean |k| of the bin's modes.
 *  nmodes: nbins int64 out (host) or NULL: the bin's mode count.
 *  stream: cudaStream_t (NULL: legacy default stream); the call returns after
 *          synchronising it.
 * The transform is cuFFT's (loaded on first use; SDOT_ERR_CUDA with a message if it
 * cannot be); the per-bin sums are 64-bit fixed point (unit 2^-38 of the bin's largest
 * |delta_k|^2), so the result is reproducible and within ~1e-10 relative of the exact
 * mean. Device scratch of about 3 M^3 doubles is allocated and freed by the call.
 */
int sdot_power_spectrum(const double* rho, int M, double L, int nbins, double* P,
                        double* kmean, int64_t* nmodes, void* stream);

/*
 * After the solve: the Kantorovich potential at tau_I on a mesh and the mass density of
 * the cells moved to an intermediate time (Sec. "Monge-Ampere-Kantorovich
 * Reconstruction": the Legendre transform of psi, and the last paragraph; Fig. 1).
 * At the context's current psi (the cells of its last evaluation at that psi; the
 * call evaluates the diagram first if needed).
 *  lambda: D(tau) / D(tau_F) in [0, 1): the Zel'dovich map q -> q + lambda (x_i - q)
 *          moves every point of cell i towards its point x_i, i.e. shrinks the cell
 *          about x_i by the factor 1 - lambda; lambda = 0 is tau_I.
 *  mesh:   M in [1, 2048] points per axis; value m = (z M + y) M + x belongs to the
 *          voxel [x, x+1] x [y, y+1] x [z, z+1] L/M and to its centre (m + 1/2) L/M.
 *  rho:    M^3 doubles out (host or device), or NULL: the mass density of the moved
 *          cells (each carries its mass nu_i uniformly), computed by exact intersection
 *          of every moved cell with the voxels; mean 1 when sum nu = |box|.
 *  phi:    M^3 doubles out, or NULL: phi_I(q) = min_i [1/2 |q - x_i|^2 - psi_i]
 *          (minimum image) at the voxel centres.
 *  owner:  M^3 int32 out, or NULL: the cell containing each voxel centre (caller
 *          order; the lowest index when the centre lies on a facet).
 * The device buffers it needs (16 M^3 bytes, plus staging for host outputs) come from
 * the context's allocator and are kept for the next call. SDOT_ERR_CAPACITY if a cell
 * cannot be rebuilt from its facets in the large polytope.
 */
int sdot_mesh(sdot_ctx* ctx, double lambda, int mesh, double* rho, double* phi,
              int32_t* owner);

/* Statistics of the context's last Laguerre evaluation (host memory out). */
int sdot_last_eval(const sdot_ctx* ctx, sdot_eval_info* info);

/* Number of seeds and kNN size of the context. */
int sdot_size(const sdot_ctx* ctx, int64_t* N, int* k);

/* Release every resource of ctx (NULL is accepted). */
void sdot_destroy(sdot_ctx* ctx);

/* Number of kernel launches this library has issued in the process so far. */
int64_t sdot_kernel_launches(void);

/* Message of the last error on the calling thread ("" if none). */
const char* sdot_last_error(void);

/*
 * Reconstruction server: jobs of different N arrive at any time and run
 * concurrently on one GPU. The paper states the problem for one box; serving many
 * boxes is this library's addition.
 *
 * Admission: jobs wait in arrival order (FIFO, no overtaking) and are admitted while
 * the sum of the admitted jobs' device footprints (sdot_server_footprint) stays
 * within hbm_budget and at most max_active jobs are admitted. An admitted job keeps
 * its whole state (positions, psi, kNN lists, facets, CSR Hessian, CG vectors)
 * resident on the device until it finishes, then its memory and slot are released
 * and the queue is admitted again. Each admitted job runs sdot_create, sdot_solve
 * and sdot_displacement on a CUDA stream and host thread of its own, so the kernels
 * of different jobs overlap on the device. With batch_clip (default), the jobs'
 * Laguerre evaluations are gathered by a batcher thread (it waits up to 0.2 ms for
 * the other running jobs) and each clipping pass runs as one persistent launch
 * over the cells of every job in the batch, pulled from one shared work counter.
 * A job's arithmetic does not depend on the other jobs: its results are the same
 * alone and in any mix.
 *
 * Job states: SDOT_JOB_QUEUED, SDOT_JOB_RUNNING, SDOT_JOB_DONE, SDOT_JOB_FAILED.
 * Times are seconds since sdot_server_create: arrival (submit), admission and
 * completion; a job's latency is completion - arrival.
 * The server functions are thread-safe.
 */
enum { SDOT_JOB_QUEUED = 0, SDOT_JOB_RUNNING = 1, SDOT_JOB_DONE = 2, SDOT_JOB_FAILED = 3 };

typedef struct sdot_server sdot_server;

typedef struct {
    size_t hbm_budget; /* device bytes the admitted jobs may hold together; 0: 90% of the
                          device memory free at creation */
    int max_active;    /* jobs admitted at once (default 8) */
    int device;        /* CUDA device ordinal; -1 (default): the current device */
    int batch_clip;    /* 1 (default): the running jobs' Laguerre evaluations are batched,
                          each clipping pass one persistent launch over the cells of all
                          of them; 0: each job launches its own passes */
} sdot_server_options;

typedef struct {
    size_t hbm_budget, used_bytes, peak_used_bytes;
    int max_active, active, peak_active;
    int64_t queued, finished, submitted;
} sdot_server_info;

/* Fill *opt with the defaults listed in sdot_server_options. */
int sdot_server_default_options(sdot_server_options* opt);

/*
 * Device bytes a job of N seeds in box holds while admitted (with options opt, NULL:
 * defaults): every array sdot_create allocates, plus a reserve of 25 Hessian entries
 * per seed (12 bytes each) for the CSR that sdot_solve builds. Host computation only.
 */
int sdot_server_footprint(int64_t N, const double box[3], const sdot_options* opt,
                          size_t* bytes);

/* Create a server (opt NULL: defaults). On error *out is NULL. */
int sdot_server_create(const sdot_server_options* opt, sdot_server** out);

/*
 * Queue a job: the solve of sdot_create(pos, mass, N, box, opt) + sdot_solve(tol)
 * + sdot_displacement. pos (N x 3) and mass (N, or NULL for uniform) must be host
 * memory; they are copied before the call returns. *id receives the job's id.
 * Returns SDOT_ERR_OOM if the job's footprint exceeds hbm_budget (it could never be
 * admitted). Errors of the solve itself are reported by sdot_server_result.
 */
int sdot_server_submit(sdot_server* srv, const double* pos, const double* mass, int64_t N,
                       const double box[3], const sdot_options* opt, double tol,
                       int64_t* id);

/* State of job id (*state: SDOT_JOB_*). */
int sdot_server_poll(sdot_server* srv, int64_t id, int* state);

/* Wait until job id has finished or timeout_s seconds passed (< 0: no limit);
 * SDOT_ERR_TIMEOUT if it has not finished. *state (may be NULL) receives its state. */
int sdot_server_wait(sdot_server* srv, int64_t id, double timeout_s, int* state);

/*
 * Collect a finished job and release its record. disp (N x 3) and psi (N) are host
 * buffers in the job's seed order, or NULL; st (may be NULL) receives the solve's
 * statistics; times (3 doubles, may be NULL) its arrival, admission and completion
 * times. Returns the job's own result code (SDOT_OK or the error of its create or
 * solve, whose message sdot_last_error() then gives on the calling thread), or
 * SDOT_ERR_NOT_READY while it is queued or running (the record is kept). disp and psi
 * are written only for a job that succeeded.
 */
int sdot_server_result(sdot_server* srv, int64_t id, double* disp, double* psi,
                       sdot_stats* st, double times[3]);

/* Occupancy and counters of the server. */
int sdot_server_get_info(sdot_server* srv, sdot_server_info* info);

/* Wait for the running jobs, drop the queued ones and release the server (NULL is
 * accepted). */
void sdot_server_destroy(sdot_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* SDOT_H */
