// Internal definitions shared by the CUDA translation units of libsdot.
// Nothing here is part of the public ABI (include/sdot.h).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "sdot.h"

namespace sdot {

// one seed position, 32-byte aligned so a load is one sector; w = caller index
struct __align__(32) Pos4 {
    double x, y, z, w;
    __host__ __device__ static Pos4 make(double x, double y, double z, double w) {
        Pos4 p;
        p.x = x;
        p.y = y;
        p.z = z;
        p.w = w;
        return p;
    }
};

// ---------------------------------------------------------------------------
// capacities
// ---------------------------------------------------------------------------
constexpr int KMAX = 64;        // largest kNN size
constexpr int MAXP = 96;        // planes of the largest polytope (6 box planes included)
constexpr int MAXT = 192;       // vertices (dual triangles) of the largest polytope
constexpr int FCAP = 64;        // facets stored per cell for the Hessian
constexpr int TOPO = 64;        // vertices of a cell's stored topology (warm start)
constexpr int CERT_NEAR = 16;   // seeds a carried security certificate re-tests exactly
constexpr int CERT_F = 6;       // floats of a certificate: ball centre (3), radius, M, w reserve
constexpr int CERT_S = 27;      // FP16 supports of a certificate (26 directions + unused centre)
constexpr int MAXLEV = 8;       // pyramid levels

// cell status bits (per cell, uint8)
enum : uint32_t {
    CS_OK = 0,
    CS_EMPTY = 1,          // polytope vanished
    CS_CAPACITY = 2,       // plane/vertex/facet/stack capacity exceeded
    CS_INCONSISTENT = 4,   // FP32 consistency check failed
    CS_UNCERTIFIED = 8,    // security test found a possible unseen cutter
    CS_TOO_LARGE = 16,     // cell reaches a non-minimum periodic image
    CS_CAP_POLY = 32,      // detail of CS_CAPACITY: planes or vertices
    CS_CAP_FACE = 64,      // detail of CS_CAPACITY: facets or vertices of one face
    CS_CAP_STACK = 128,    // detail of CS_CAPACITY: traversal stack
};

// ---------------------------------------------------------------------------
// device data of one context (all arrays in grid-sorted seed order unless noted)
// ---------------------------------------------------------------------------
struct Pyramid {
    int nlev;
    int dim[MAXLEV][3];       // nodes per axis at each level (level 0 = grid cells)
    int64_t off[MAXLEV];      // offset of each level in psimax
    float* psimax;            // upper bound of psi/a^2 over the node (rounded up)
};

struct Grid {
    int G[3];                 // grid cells per axis
    double h[3];              // cell size per axis (absolute units)
    int64_t ncell;
    int32_t* cell_start;      // ncell + 1
};

struct DeviceState {
    int64_t N;
    int k;
    double L[3];
    double a;                 // length unit: (|box| / N)^(1/3)
    // seeds
    Pos4* pos;             // sorted positions; w = caller index (exact in fp64)
    float4* posf;             // (offset in grid cell / a, psi/a^2 hi), per evaluation
    float* pslo;              // psi/a^2 lo part (psi/a^2 = hi + lo)
    uint4* ioff;              // offset in the grid cell as 32-bit fixed point (x, y, z, 0)
    int32_t* leafc;           // grid cell of each seed: x | y << 10 | z << 20
    int facets_valid;         // fcnt/fcol hold a complete previous diagram
    int carry = 1;            // carry security certificates between evaluations
    int32_t* perm;            // sorted -> caller index
    int32_t* iperm;           // caller -> sorted index
    double* nu;               // masses (sorted)
    double* psi;              // current psi (sorted)
    double* psi_trial;        // line-search trial (sorted)
    double* delta;            // Newton direction (sorted)
    int32_t* knn;             // N * k sorted neighbour indices
    double* knn_d2k;          // d^2 of the k-th neighbour (key of the seen set)
    // cell outputs of the last evaluation
    double* vol;              // N
    double* m1;               // N * 3, int_{V} (q - y) dq  (absolute units)
    float* anchor;            // N * 3, previous local centroid / a (traversal anchor)
    uint8_t* status;          // N
    int32_t* fcnt;            // N facet counts
    int32_t* fcol;            // N * FCAP facet neighbours (sorted index)
    double* fval;             // N * FCAP facet coefficients A/|d|
    uint32_t* topo;           // N * TOPO vertices of each cell as three plane indices
                              // (0..5 box faces, 6 + k facet k of fcol)
    uint8_t* topo_n;          // N vertex counts of topo (0: none stored)
    // security certificates carried between evaluations (see process_cell): per cell the
    // ball and reserves, the inflated supports, the seeds to re-test and their count
    // (0xff: none); psi of the previous evaluation, for the change of psi since
    float* cert_f;            // N * CERT_F
    uint16_t* cert_s;         // N * CERT_S (FP16 bits, rounded up)
    int32_t* cert_j;          // N * CERT_NEAR
    uint8_t* cert_n;          // N
    double* psi_prev;         // N
    int32_t* queue;           // N, re-queued cells
    int32_t* queue64;         // N, cells for the FP64 re-clip
    int32_t* counters;        // [0] requeue count [1] fp64 count [2] work counter
                              // [3] error flags [4] work counter 2 [5] work counter 3
                              // [8..24) 64-bit diagnostic work counters
    // CSR (sorted order)
    int64_t* row_ptr;         // N + 1
    int32_t* col;             // nnz capacity N * (FCAP + 1)
    double* val;
    int32_t* rowcnt;          // N (+1 pad)
    // CSR (caller order), built on demand for sdot_laguerre
    int64_t* row_ptr_u;
    int32_t* col_u;
    double* val_u;
    // CG vectors (x: the Newton direction, z: u = M^-1 r, q: w = L u, sv: s = L p)
    double *x, *r, *z, *p, *q, *sv, *dinv;
    float* uf;                // u rounded to FP32, the operand the SpMV gathers
    // the Newton matrix L in sliced-ELL form (slices of 32 rows, entry k of row
    // 32 l + m at sell_ptr[l] + 32 k + m, columns ascending within a row): neighbour
    // column and FP32 weight A/|d|; the diagonal is implied (zero row sums)
    int64_t* sell_ptr;        // nslice + 1
    int32_t* sell_w;          // nslice + 1 slice widths (scan input)
    int32_t* sell_col;
    float* sell_val;
    double* partials;         // reduction partials
    double* scal;             // device scalars
    Grid grid;
    Pyramid pyr;
};

// NVTX range for the lifetime of the object (phases of the hot path, visible to
// profilers; a no-op when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);

#define SDOT_CUDA_TRY(expr)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::sdot::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));       \
            return SDOT_ERR_CUDA;                                                        \
        }                                                                                \
    } while (0)

// ---------------------------------------------------------------------------
// launchers (host functions defined in the .cu files)
// ---------------------------------------------------------------------------
int num_sms();

// process-wide count of kernel launches issued by this library
void note_launch();
unsigned long long launch_count();

// exclusive scans (in may alias out); temp must hold scan_temp_elems(n) elements
size_t scan_temp_bytes(int64_t n);
int scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* temp,
                              cudaStream_t s);
int scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, void* temp,
                       cudaStream_t s);

// grid_knn.cu
// who: the public entry point, named in the error message
int build_grid(DeviceState& d, const double* pos_user_dev, double seeds_per_leaf,
               void* temp, cudaStream_t s, const char* who);
int build_knn(DeviceState& d, cudaStream_t s, int* dup_flag_host);
int knn_to_user(const DeviceState& d, int32_t* out_user_dev, cudaStream_t s);

// clip.cu
struct EvalResult {
    double sum_vol, max_rel_err, l2_err, min_vol;
    int64_t requeued, reclipped, n_empty;
    uint32_t flags;
    float ms;
    float ms_pass[3];             // certify pass, re-queue pass, FP64 re-clip pass
    unsigned long long work[8];   // diagnostic work counters (zero unless compiled in)
    int64_t carried = 0;          // cells certified by a carried certificate (pass 1)
};
int build_pyramid(DeviceState& d, const double* psi, cudaStream_t s);
int evaluate_cells(DeviceState& d, const double* psi, int precision, EvalResult* res,
                   cudaStream_t s);
// Batched evaluation of n contexts (one persistent launch per pass for all of their
// cells; results identical to evaluate_cells on each context). The scratch holds the
// job tables for up to cap contexts.
struct BatchScratch;
int batch_scratch_create(int cap, BatchScratch** out);
void batch_scratch_destroy(BatchScratch* b);
int evaluate_cells_batch(DeviceState* const* ds, const double* const* psis, const int* precs,
                         EvalResult* res, int n, BatchScratch* sc, cudaStream_t s);
// evaluation hook of a context (the server's batcher): replaces evaluate_cells
typedef int (*EvalHook)(void* user, DeviceState* d, const double* psi, int precision,
                        EvalResult* res, cudaStream_t s);

// mesh.cu: phi_I and owners at the M^3 mesh points and the mass density of the cells
// moved by lambda (any output may be null); scratch holds 16 M^3 bytes
int mesh_eval(DeviceState& d, int M, double lambda, double* rho_dev, double* phi_dev,
              int32_t* owner_dev, void* scratch, cudaStream_t s);

// linalg.cu
int csr_count(DeviceState& d, int64_t* nnz_out, cudaStream_t s);  // row_ptr and nnz
int csr_fill(DeviceState& d, cudaStream_t s);                      // col, val, dinv
int assemble_csr_user(DeviceState& d, int64_t nnz, cudaStream_t s);
// sliced-ELL Newton matrix: sell_build counts (sell_ptr in slice widths, *entries the
// storage it needs), sell_fill writes it (arrays of that capacity) and dinv
int sell_build(DeviceState& d, int64_t* entries, int64_t* offdiag, cudaStream_t s);
int sell_fill(DeviceState& d, cudaStream_t s);
// Jacobi-preconditioned CG on L x = (nu - V) - mean, until ||r|| <= rtol ||r0||
int cg_solve(DeviceState& d, double rtol, int maxit, int* iters, double* rel_res,
             cudaStream_t s);
int axpy_gauge(DeviceState& d, const double* psi, const double* delta, double alpha,
               double* out, cudaStream_t s);
int subtract_mean(DeviceState& d, double* v, cudaStream_t s);
int scatter_to_user(const DeviceState& d, const double* sorted, double* user, int width,
                    cudaStream_t s);
int gather_from_user(const DeviceState& d, const double* user, double* sorted, int width,
                     cudaStream_t s);
int centroids_user(const DeviceState& d, double* out_user, int wrap_abs, cudaStream_t s);
int status_to_user(const DeviceState& d, uint8_t* out_user, cudaStream_t s);
int check_masses(const DeviceState& d, double* sum_out, double* min_out, cudaStream_t s);
// *ok = every v[i], i < n (device memory), is finite; synchronises s
int all_finite(DeviceState& d, const double* v, int64_t n, bool* ok, cudaStream_t s);

// sdot_create with all work on stream (api.cu)
int create_context(const double* pos, const double* mass, int64_t N, const double box[3],
                   const sdot_options* opt, cudaStream_t stream, sdot_ctx** out);
// device bytes a context for N seeds holds, CSR reserve included (api.cu)
int context_footprint(int64_t N, const double box[3], const sdot_options* opt, size_t* bytes);
// route the context's evaluations through hook (null: evaluate_cells) (api.cu)
void set_eval_hook(sdot_ctx* c, EvalHook hook, void* user);

}  // namespace sdot
