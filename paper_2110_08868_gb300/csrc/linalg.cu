// Hessian assembly (CSR) and the Newton linear solve.
//
// The second derivative of K (eq. SDK; K is C^2 by the smoothness paragraph of Sec.
// "Monge-Ampere-Kantorovich Reconstruction") is -L with L the weighted graph
// Laplacian of the Laguerre diagram: L_ij = -A_ij/|d_ij| for every facet, L_ii =
// -sum_j L_ij. Each cell reports its own facets; the matrix keeps the mean of the
// two reports of a facet and drops facets seen by one side only (zero-area contacts
// resolved differently by rounding), so L is exactly symmetric with zero row sums.
//
// The Newton direction solves L delta = nu - V (projected to mean zero: L is
// singular with the constants as kernel) by Jacobi-preconditioned conjugate
// gradients. Dot products use fixed-order two-level reductions (per-block partials
// summed in block order by every consumer) so results are bitwise reproducible.
#include <math.h>

#include "internal.cuh"

namespace sdot {

#define FULLMASK 0xffffffffu

// ---------------------------------------------------------------------------
// CSR assembly
// ---------------------------------------------------------------------------
// Symmetrised coefficient of facet t of cell i, or 0 when it must not enter the
// matrix: the first occurrence of column j in row i carries the whole pair
// 1/2 (sum of cell i's reports of j + sum of cell j's reports of i); later duplicate
// occurrences and facets reported by one side only give 0. L is therefore exactly
// symmetric even when a cell reports a neighbour twice.
__device__ __forceinline__ double sym_value(const int32_t* __restrict__ fcnt,
                                            const int32_t* __restrict__ fcol,
                                            const double* __restrict__ fval, int64_t i, int t) {
    const int32_t j = fcol[i * FCAP + t];
    for (int u = 0; u < t; u++)
        if (fcol[i * FCAP + u] == j) return 0.0;  // not the first occurrence
    double cij = 0.0;
    const int ni = fcnt[i];
    for (int u = t; u < ni; u++)
        if (fcol[i * FCAP + u] == j) cij += fval[i * FCAP + u];
    double cji = 0.0;
    bool seen = false;
    const int nj = fcnt[j];
    for (int u = 0; u < nj; u++)
        if (fcol[(int64_t)j * FCAP + u] == (int32_t)i) {
            cji += fval[(int64_t)j * FCAP + u];
            seen = true;
        }
    return seen ? 0.5 * (cij + cji) : 0.0;
}

// Row i's facets, one per lane (rows of at most 32 facets): the symmetrised
// coefficient of each first occurrence of a column (sym_value's value, with the same
// sums in the same order, so L stays exactly symmetric) and whether it enters L.
struct RowSym {
    int32_t j;
    double v;
    bool keep;
};

__device__ __forceinline__ RowSym row_sym_warp(const int32_t* __restrict__ fcnt,
                                               const int32_t* __restrict__ fcol,
                                               const double* __restrict__ fval, int64_t i,
                                               int n, int lane) {
    RowSym r;
    const bool act = lane < n;
    r.j = act ? fcol[i * FCAP + lane] : -1;
    const double f = act ? fval[i * FCAP + lane] : 0.0;
    // lanes holding the same column; inactive lanes get keys of their own
    const uint32_t mm = __match_any_sync(FULLMASK, act ? (uint32_t)r.j : 0x80000000u | lane);
    const bool first = act && (__ffs(mm) - 1) == lane;
    // i's reports of j, summed in slot order from the first occurrence (as sym_value)
    double cij = 0.0 + f;
    if (__any_sync(FULLMASK, __popc(mm) > 1)) {
        cij = 0.0;
        for (int src = 0; src < 32; src++) {
            const double fs = __shfl_sync(FULLMASK, f, src);
            if ((mm >> src) & 1u) cij += fs;
        }
    }
    double cji = 0.0;
    bool seen = false;
    if (first) {
        const int nj = fcnt[r.j];
        for (int u = 0; u < nj; u++)
            if (fcol[(int64_t)r.j * FCAP + u] == (int32_t)i) {
                cji += fval[(int64_t)r.j * FCAP + u];
                seen = true;
            }
    }
    r.v = (first && seen) ? 0.5 * (cij + cji) : 0.0;
    r.keep = r.v > 0.0;
    return r;
}

// one warp per row: the row's entry count (kept facets + the diagonal)
__global__ void csr_count_kernel(const int32_t* __restrict__ fcnt, const int32_t* __restrict__ fcol,
                                 const double* __restrict__ fval, int64_t N,
                                 int32_t* __restrict__ rowcnt) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= N) return;
    const int n = fcnt[i];
    if (n > 32) {  // rare: the row in lane 0, serially
        if (lane == 0) {
            int kept = 0;
            for (int t = 0; t < n; t++)
                if (sym_value(fcnt, fcol, fval, i, t) > 0.0) kept++;
            rowcnt[i] = kept + 1;
        }
        return;
    }
    const RowSym r = row_sym_warp(fcnt, fcol, fval, i, n, lane);
    const uint32_t km = __ballot_sync(FULLMASK, r.keep);
    if (lane == 0) rowcnt[i] = __popc(km) + 1;
}

// one warp per row: the diagonal first, then the kept entries in increasing column
// (each lane's rank among them), values -c_ij; the diagonal is their warp sum
__global__ void csr_fill_kernel(const int32_t* __restrict__ fcnt, const int32_t* __restrict__ fcol,
                                const double* __restrict__ fval, int64_t N,
                                const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                                double* __restrict__ val, double* __restrict__ dinv) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= N) return;
    const int n = fcnt[i];
    const int64_t p0 = row_ptr[i];
    if (n > 32) {  // rare: the row in lane 0, serially (insertion by column)
        if (lane == 0) {
            int64_t p = p0 + 1;
            double diag = 0.0;
            for (int t = 0; t < n; t++) {
                const double v = sym_value(fcnt, fcol, fval, i, t);
                if (!(v > 0.0)) continue;
                const int32_t j = fcol[i * FCAP + t];
                int64_t q = p;
                while (q > p0 + 1 && col[q - 1] > j) {
                    col[q] = col[q - 1];
                    val[q] = val[q - 1];
                    q--;
                }
                col[q] = j;
                val[q] = -v;
                p++;
                diag += v;
            }
            col[p0] = (int32_t)i;
            val[p0] = diag;
            dinv[i] = diag > 0.0 ? 1.0 / diag : 0.0;
        }
        return;
    }
    const RowSym r = row_sym_warp(fcnt, fcol, fval, i, n, lane);
    const uint32_t km = __ballot_sync(FULLMASK, r.keep);
    int rank = 0;
    for (int src = 0; src < 32; src++) {
        const int32_t js = __shfl_sync(FULLMASK, r.j, src);
        if (((km >> src) & 1u) && js < r.j) rank++;
    }
    if (r.keep) {
        col[p0 + 1 + rank] = r.j;
        val[p0 + 1 + rank] = -r.v;
    }
    double diag = r.keep ? r.v : 0.0;
    for (int o = 16; o > 0; o >>= 1) diag += __shfl_xor_sync(FULLMASK, diag, o);
    if (lane == 0) {
        col[p0] = (int32_t)i;
        val[p0] = diag;
        dinv[i] = diag > 0.0 ? 1.0 / diag : 0.0;
    }
}

int csr_count(DeviceState& d, int64_t* nnz_out, cudaStream_t s) {
    const int64_t N = d.N;
    unsigned nb = (unsigned)((N + 7) / 8);  // 8 rows (warps) per block
    csr_count_kernel<<<nb, 256, 0, s>>>(d.fcnt, d.fcol, d.fval, N, d.rowcnt);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    // row_ptr = exclusive scan over N+1 entries (rowcnt[N] == 0)
    SDOT_CUDA_TRY(cudaMemsetAsync(d.rowcnt + N, 0, 4, s));
    int rc = scan_exclusive_i32_to_i64(d.rowcnt, d.row_ptr, N + 1, d.partials + 65536, s);
    if (rc) return rc;
    int64_t nnz = 0;
    SDOT_CUDA_TRY(cudaMemcpyAsync(&nnz, d.row_ptr + N, 8, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    *nnz_out = nnz;
    return SDOT_OK;
}

int csr_fill(DeviceState& d, cudaStream_t s) {
    const int64_t N = d.N;
    unsigned nb = (unsigned)((N + 7) / 8);  // 8 rows (warps) per block
    csr_fill_kernel<<<nb, 256, 0, s>>>(d.fcnt, d.fcol, d.fval, N, d.row_ptr, d.col, d.val, d.dinv);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

// the same matrix in the caller's index order
__global__ void csr_user_count(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ perm,
                               int64_t N, int32_t* __restrict__ cnt_user) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    cnt_user[perm[s]] = (int32_t)(row_ptr[s + 1] - row_ptr[s]);
}

// one warp per sorted row s: row perm[s] of the caller's matrix, the diagonal first and
// the off-diagonal entries ranked by their caller-order column
__global__ void csr_user_fill(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const int32_t* __restrict__ perm,
                              int64_t N, const int64_t* __restrict__ rp_u,
                              int32_t* __restrict__ col_u, double* __restrict__ val_u) {
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= N) return;
    const int64_t b = row_ptr[s], e = row_ptr[s + 1];
    const int64_t o = rp_u[perm[s]];
    const int m = (int)(e - b) - 1;  // off-diagonal entries
    if (lane == 0) {
        col_u[o] = perm[col[b]];
        val_u[o] = val[b];
    }
    if (m > 32) {  // rare: lane 0, insertion by column
        if (lane == 0) {
            int64_t p = o + 1;
            for (int64_t t = b + 1; t < e; t++) {
                const int32_t j = perm[col[t]];
                const double v = val[t];
                int64_t q = p;
                while (q > o + 1 && col_u[q - 1] > j) {
                    col_u[q] = col_u[q - 1];
                    val_u[q] = val_u[q - 1];
                    q--;
                }
                col_u[q] = j;
                val_u[q] = v;
                p++;
            }
        }
        return;
    }
    const bool act = lane < m;
    const int32_t j = act ? perm[col[b + 1 + lane]] : 0;
    const double v = act ? val[b + 1 + lane] : 0.0;
    int rank = 0;
    for (int src = 0; src < 32; src++) {
        const int32_t js = __shfl_sync(FULLMASK, j, src);
        if (src < m && js < j) rank++;
    }
    if (act) {
        col_u[o + 1 + rank] = j;
        val_u[o + 1 + rank] = v;
    }
}

int assemble_csr_user(DeviceState& d, int64_t nnz, cudaStream_t s) {
    (void)nnz;
    const int64_t N = d.N;
    unsigned nb = (unsigned)((N + 255) / 256);
    csr_user_count<<<nb, 256, 0, s>>>(d.row_ptr, d.perm, N, d.rowcnt);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    SDOT_CUDA_TRY(cudaMemsetAsync(d.rowcnt + N, 0, 4, s));
    int rc = scan_exclusive_i32_to_i64(d.rowcnt, d.row_ptr_u, N + 1, d.partials + 65536, s);
    if (rc) return rc;
    csr_user_fill<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(d.row_ptr, d.col, d.val, d.perm, N,
                                                         d.row_ptr_u, d.col_u, d.val_u);
                                     note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

// ---------------------------------------------------------------------------
// Newton system: sliced-ELL matrix and conjugate gradients
// ---------------------------------------------------------------------------
constexpr int CG_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int u = 0; u < (int)(blockDim.x >> 5); u++) t += sh[u];
    return t;  // valid in thread 0
}

// Off-diagonal entries kept per row (symmetrised facets of positive weight); one warp
// per slice of 32 rows, whose width (longest row) it records, and the total count.
__global__ void sell_count_kernel(const int32_t* __restrict__ fcnt, const int32_t* __restrict__ fcol,
                                  const double* __restrict__ fval, int64_t N, int64_t nslice,
                                  int32_t* __restrict__ width, unsigned long long* __restrict__ nnz) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long tot = 0;
    for (int64_t sl = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sl < nslice;
         sl += nw) {
        const int64_t i = sl * 32 + lane;
        int kept = 0;
        if (i < N) {
            const int n = fcnt[i];
            for (int t = 0; t < n; t++)
                if (sym_value(fcnt, fcol, fval, i, t) > 0.0) kept++;
        }
        const int w = __reduce_max_sync(FULLMASK, kept);
        if (lane == 0) width[sl] = w;
        tot += (unsigned long long)__reduce_add_sync(FULLMASK, (unsigned)kept);
    }
    if (lane == 0 && tot) atomicAdd(nnz, tot);
}

// The entries of each slice column by column (entry k of row 32 sl + l at
// ptr[sl] + 32 k + l), each row in increasing column order, padded with zero weights
// on the row's own column. Weights are stored in FP32 in both precisions (the SpMV
// works in FP32 per entry); the Jacobi inverse diagonal is taken from the stored
// weights, so the stored matrix has exactly zero row sums.
__global__ void sell_fill_kernel(const int32_t* __restrict__ fcnt, const int32_t* __restrict__ fcol,
                                 const double* __restrict__ fval, int64_t N, int64_t nslice,
                                 const int64_t* __restrict__ ptr, int32_t* __restrict__ col,
                                 float* __restrict__ val, double* __restrict__ dinv) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t sl = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sl < nslice;
         sl += nw) {
        const int64_t i = sl * 32 + lane;
        const int64_t base = ptr[sl] + lane;
        const int w = (int)((ptr[sl + 1] - ptr[sl]) >> 5);
        int k = 0;
        double diag = 0.0;
        if (i < N) {
            const int n = fcnt[i];
            for (int t = 0; t < n && k < w; t++) {
                const double v = sym_value(fcnt, fcol, fval, i, t);
                if (!(v > 0.0)) continue;
                const float vt = (float)v;
                const int32_t c = fcol[i * FCAP + t];
                // insertion by column: entry k of neighbouring rows then lies near the
                // same stencil direction, so the gathers of a warp share cache lines
                int b = k;
                for (; b > 0; b--) {
                    const int32_t cb = col[base + 32 * (int64_t)(b - 1)];
                    if (cb <= c) break;
                    col[base + 32 * (int64_t)b] = cb;
                    val[base + 32 * (int64_t)b] = val[base + 32 * (int64_t)(b - 1)];
                }
                col[base + 32 * (int64_t)b] = c;
                val[base + 32 * (int64_t)b] = vt;
                diag += (double)vt;
                k++;
            }
            dinv[i] = diag > 0.0 ? 1.0 / diag : 0.0;
        }
        const int32_t self = i < N ? (int32_t)i : 0;
        for (; k < w; k++) {
            col[base + 32 * (int64_t)k] = self;
            val[base + 32 * (int64_t)k] = 0.f;
        }
    }
}

// Chronopoulos-Gear form of Jacobi-preconditioned CG (one reduction point per
// iteration): with u = M^-1 r, w = L u, gamma = (r, u), delta = (w, u),
//   beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
//   (first iteration: beta = 0, alpha = gamma / delta),
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s.
// The SpMV kernel computes w and the partials of delta; its last block to finish
// (counter + fence, no waiting) sums the partials of delta and of the gamma and (r, r)
// left by the update kernel, in block order, and writes the scalars. Scalars in
// cg[]: 0 alpha, 1 beta, 2 gamma_old, 3 alpha_old, 4 (r, r), 5 first-iteration flag.
__global__ void cg_init_kernel(const double* __restrict__ nu, const double* __restrict__ vol,
                               double mean, const double* __restrict__ dinv, int64_t N,
                               double* __restrict__ x, double* __restrict__ r,
                               double* __restrict__ u, float* __restrict__ uf,
                               double* __restrict__ p, double* __restrict__ sv,
                               double* __restrict__ part, double* __restrict__ cg) {
    __shared__ double sh[32];
    double g = 0, rr = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = (nu[i] - vol[i]) - mean;
        const double ui = dinv[i] * ri;
        x[i] = 0.0;
        r[i] = ri;
        u[i] = ui;
        uf[i] = (float)ui;
        p[i] = 0.0;
        sv[i] = 0.0;
        g += ri * ui;
        rr += ri * ri;
    }
    const double a = block_sum(g, sh);
    const double b = block_sum(rr, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = a;
        part[3 * blockIdx.x + 2] = b;
        if (blockIdx.x == 0) cg[5] = 1.0;
    }
}

// w = L u in the Laplacian form (L u)_i = sum_j c_ij (u_i - u_j). Every stored entry
// costs two FP32 operations on the FP32 copy of u: GB300 issues FP64 at about two
// operations per clock per SM, so FP64 arithmetic per entry, not HBM, bounded this
// loop. A row's sum is rounded to FP64 once. The error of w is that of FP32 products
// (about 1e-7 of sum_j c_ij (|u_i| + |u_j|)), far below the relative residual the
// Newton direction is solved to, and the stored matrix keeps its exact zero row sums.
__global__ void __launch_bounds__(CG_THREADS, 8)
    cg_spmv_kernel(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                   const float* __restrict__ val, int64_t N, int64_t nslice,
                   const float* __restrict__ uf, const double* __restrict__ u,
                   double* __restrict__ w, double* __restrict__ part,
                   unsigned int* __restrict__ done, double* __restrict__ cg) {
    __shared__ double sh[32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    double dl = 0.0;
    for (int64_t sl = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sl < nslice;
         sl += nw) {
        const int64_t i = sl * 32 + lane;
        const int64_t b0 = ptr[sl];
        const int wd = (int)((ptr[sl + 1] - b0) >> 5);
        const float ui = i < N ? uf[i] : 0.f;
        float acc = 0.f;
        const int32_t* cp = col + b0 + lane;
        const float* vp = val + b0 + lane;
        int k = 0;
        for (; k + 8 <= wd; k += 8) {
            int32_t j[8];
            float c[8], v[8];
#pragma unroll
            for (int e = 0; e < 8; e++) {
                j[e] = cp[32 * e];
                c[e] = vp[32 * e];
            }
#pragma unroll
            for (int e = 0; e < 8; e++) v[e] = uf[j[e]];
#pragma unroll
            for (int e = 0; e < 8; e++) acc = fmaf(c[e], ui - v[e], acc);
            cp += 256;
            vp += 256;
        }
        for (; k < wd; k++) {
            acc = fmaf(vp[0], ui - uf[cp[0]], acc);
            cp += 32;
            vp += 32;
        }
        if (i < N) {
            const double wi = (double)acc;
            w[i] = wi;
            dl += wi * u[i];
        }
    }
    const double a = block_sum(dl, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 1] = a;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block: fixed-order sums of the partials, then the scalars
    __threadfence();
    double sg = 0, sd = 0, sr = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        sg += __ldcg(&part[3 * b + 0]);
        sd += __ldcg(&part[3 * b + 1]);
        sr += __ldcg(&part[3 * b + 2]);
    }
    const double G = block_sum(sg, sh);
    const double D = block_sum(sd, sh);
    const double RR = block_sum(sr, sh);
    if (threadIdx.x == 0) {
        double alpha, beta;
        if (cg[5] != 0.0) {
            beta = 0.0;
            alpha = D != 0.0 ? G / D : 0.0;
        } else {
            beta = cg[2] != 0.0 ? G / cg[2] : 0.0;
            const double den = D - beta * G / cg[3];
            alpha = den != 0.0 ? G / den : 0.0;
        }
        cg[0] = alpha;
        cg[1] = beta;
        cg[2] = G;
        cg[3] = alpha;
        cg[4] = RR;
        cg[5] = 0.0;
        *done = 0u;
    }
}

__global__ void cg_update_kernel(const double* __restrict__ cg, const double* __restrict__ dinv,
                                 int64_t N, const double* __restrict__ w, double* __restrict__ p,
                                 double* __restrict__ sv, double* __restrict__ x,
                                 double* __restrict__ r, double* __restrict__ u,
                                 float* __restrict__ uf, double* __restrict__ part) {
    __shared__ double sh[32];
    const double alpha = __ldcg(&cg[0]), beta = __ldcg(&cg[1]);
    double g = 0, rr = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double pi = u[i] + beta * p[i];
        const double si = w[i] + beta * sv[i];
        const double ri = r[i] - alpha * si;
        const double ui = dinv[i] * ri;
        p[i] = pi;
        sv[i] = si;
        x[i] += alpha * pi;
        r[i] = ri;
        u[i] = ui;
        uf[i] = (float)ui;
        g += ri * ui;
        rr += ri * ri;
    }
    const double a = block_sum(g, sh);
    const double b = block_sum(rr, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = a;
        part[3 * blockIdx.x + 2] = b;
    }
}

__global__ void partial_sum_kernel(const double* __restrict__ part, int nb, int stride, int off,
                                   double* __restrict__ out) {
    __shared__ double sh[32];
    double v = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[(int64_t)b * stride + off];
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) *out = t;
}

int sell_build(DeviceState& d, int64_t* entries, int64_t* offdiag, cudaStream_t s) {
    const int64_t N = d.N;
    const int64_t nslice = (N + 31) / 32;
    const int nb = 8 * num_sms();
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(d.scal + 40);
    SDOT_CUDA_TRY(cudaMemsetAsync(cnt, 0, 8, s));
    sell_count_kernel<<<nb, CG_THREADS, 0, s>>>(d.fcnt, d.fcol, d.fval, N, nslice, d.sell_w, cnt);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    SDOT_CUDA_TRY(cudaMemsetAsync(d.sell_w + nslice, 0, 4, s));
    int rc = scan_exclusive_i32_to_i64(d.sell_w, d.sell_ptr, nslice + 1, d.partials + 65536, s);
    if (rc) return rc;
    int64_t h[2] = {0, 0};
    SDOT_CUDA_TRY(cudaMemcpyAsync(&h[0], d.sell_ptr + nslice, 8, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaMemcpyAsync(&h[1], cnt, 8, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    *entries = 32 * h[0];  // slice widths sum to h[0]; each slice holds 32 rows
    *offdiag = h[1];
    return SDOT_OK;
}

__global__ void scale_ptr_kernel(int64_t* __restrict__ ptr, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) ptr[t] *= 32;
}

int sell_fill(DeviceState& d, cudaStream_t s) {
    const int64_t N = d.N;
    const int64_t nslice = (N + 31) / 32;
    const int nb = 8 * num_sms();
    scale_ptr_kernel<<<(unsigned)((nslice + 1 + 255) / 256), 256, 0, s>>>(d.sell_ptr, nslice + 1);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    sell_fill_kernel<<<nb, CG_THREADS, 0, s>>>(d.fcnt, d.fcol, d.fval, N, nslice, d.sell_ptr,
                                               d.sell_col, d.sell_val, d.dinv);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

// Blocks per SM that the CG kernels can all keep resident at once. The SpMV and the
// update share the per-block partials, so they run on one grid, and that grid is a
// single wave: a second, partial wave would run its share of the rows at a fraction
// of the occupancy.
static int cg_blocks_per_sm() {
    static int cached = 0;
    if (cached) return cached;
    int b = 8, o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, cg_spmv_kernel, CG_THREADS, 0) ==
            cudaSuccess && o > 0)
        b = o < b ? o : b;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, cg_update_kernel, CG_THREADS, 0) ==
            cudaSuccess && o > 0)
        b = o < b ? o : b;
    cudaGetLastError();
    cached = b;
    return b;
}

int cg_solve(DeviceState& d, double rtol, int maxit, int* iters, double* rel_res,
             cudaStream_t s) {
    NvtxRange nv("cg");
    const int64_t N = d.N;
    const int64_t nslice = (N + 31) / 32;
    // memory-bound loops, one resident wave of 256-thread blocks
    const int nb = cg_blocks_per_sm() * num_sms();
    double* part = d.partials;  // 3 per block
    double* cg = d.scal + 16;   // scalars (see cg_spmv_kernel)
    unsigned int* done = reinterpret_cast<unsigned int*>(d.scal + 32);
    double* hs = d.scal + 8;
    // mean of g = nu - V (its sum is rounding noise when sum nu = |box|), from the last
    // evaluation's reduction: scal[0] holds sum V
    double sums[1];
    SDOT_CUDA_TRY(cudaMemcpyAsync(sums, d.scal, 8, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    const double box = d.L[0] * d.L[1] * d.L[2];
    const double mean = (box - sums[0]) / (double)N;
    SDOT_CUDA_TRY(cudaMemsetAsync(done, 0, sizeof(unsigned int), s));
    cg_init_kernel<<<nb, CG_THREADS, 0, s>>>(d.nu, d.vol, mean, d.dinv, N, d.x, d.r, d.z, d.uf,
                                             d.p, d.sv, part, cg);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    partial_sum_kernel<<<1, CG_THREADS, 0, s>>>(part, nb, 3, 2, hs);
    note_launch();
    double h = 0;
    SDOT_CUDA_TRY(cudaMemcpyAsync(&h, hs, 8, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    const double rr0 = h;
    *iters = 0;
    *rel_res = 0.0;
    if (!(rr0 > 0.0)) return SDOT_OK;
    const double thr = rtol * rtol * rr0;
    const int check = 8;
    int it = 0;
    double rr = rr0;
    // u lives in d.z and w in d.q
    while (it < maxit) {
        for (int c = 0; c < check && it < maxit; c++, it++) {
            cg_spmv_kernel<<<nb, CG_THREADS, 0, s>>>(d.sell_ptr, d.sell_col, d.sell_val, N, nslice,
                                                     d.uf, d.z, d.q, part, done, cg);
            note_launch();
            cg_update_kernel<<<nb, CG_THREADS, 0, s>>>(cg, d.dinv, N, d.q, d.p, d.sv, d.x, d.r,
                                                       d.z, d.uf, part);
            note_launch();
        }
        SDOT_CUDA_TRY(cudaGetLastError());
        // (r, r) after the last update
        partial_sum_kernel<<<1, CG_THREADS, 0, s>>>(part, nb, 3, 2, hs);
        note_launch();
        SDOT_CUDA_TRY(cudaMemcpyAsync(&h, hs, 8, cudaMemcpyDeviceToHost, s));
        SDOT_CUDA_TRY(cudaStreamSynchronize(s));
        rr = h;
        if (!(rr > thr)) break;
    }
    *iters = it;
    *rel_res = sqrt(rr / rr0);
    return SDOT_OK;
}

// ---------------------------------------------------------------------------
// vector helpers
// ---------------------------------------------------------------------------
__global__ void axpy_kernel(const double* __restrict__ a, const double* __restrict__ b,
                            double alpha, int64_t N, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = a[i] + alpha * b[i];
}

int axpy_gauge(DeviceState& d, const double* psi, const double* delta, double alpha, double* out,
               cudaStream_t s) {
    axpy_kernel<<<(unsigned)((d.N + 255) / 256), 256, 0, s>>>(psi, delta, alpha, d.N, out);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

__global__ void sum_kernel(const double* __restrict__ v, int64_t N, double* __restrict__ part) {
    __shared__ double sh[32];
    double t = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        t += v[i];
    double a = block_sum(t, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// fixed-order sum of nb partials with stride; every block gets the same value
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int nb, int stride,
                                               double* sh) {
    double v = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[(int64_t)b * stride];
    const double t = block_sum(v, sh);
    __shared__ double bc;
    if (threadIdx.x == 0) bc = t;
    __syncthreads();
    return bc;
}

__global__ void sub_mean_kernel(double* __restrict__ v, int64_t N, const double* __restrict__ part,
                                int nb) {
    __shared__ double sh[32];
    double m = sum_partials(part, nb, 1, sh) / (double)N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] -= m;
}

int subtract_mean(DeviceState& d, double* v, cudaStream_t s) {
    const int nb = 2 * num_sms();
    sum_kernel<<<nb, 256, 0, s>>>(v, d.N, d.partials);
    note_launch();
    sub_mean_kernel<<<nb, 256, 0, s>>>(v, d.N, d.partials, nb);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

__global__ void scatter_kernel_w(const double* __restrict__ in, const int32_t* __restrict__ perm,
                                 int64_t N, int w, double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * w) return;
    int64_t s = t / w;
    int c = (int)(t - s * w);
    out[(int64_t)perm[s] * w + c] = in[t];
}

__global__ void gather_kernel_w(const double* __restrict__ in, const int32_t* __restrict__ perm,
                                int64_t N, int w, double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * w) return;
    int64_t s = t / w;
    int c = (int)(t - s * w);
    out[t] = in[(int64_t)perm[s] * w + c];
}

int scatter_to_user(const DeviceState& d, const double* sorted, double* user, int w,
                    cudaStream_t s) {
    int64_t n = d.N * w;
    scatter_kernel_w<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sorted, d.perm, d.N, w, user);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

int gather_from_user(const DeviceState& d, const double* user, double* sorted, int w,
                     cudaStream_t s) {
    int64_t n = d.N * w;
    gather_kernel_w<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(user, d.perm, d.N, w, sorted);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

// wrap_abs = 1: absolute centroid wrapped into the box; 0: displacement y - c = -m1/V
__global__ void centroid_kernel(const Pos4* __restrict__ pos, const double* __restrict__ m1,
                                const double* __restrict__ vol, const int32_t* __restrict__ perm,
                                int64_t N, double Lx, double Ly, double Lz, int wrap_abs,
                                double* __restrict__ out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    double v = vol[s];
    double c[3] = {0, 0, 0};
    if (v > 0) {
        c[0] = m1[3 * s] / v;
        c[1] = m1[3 * s + 1] / v;
        c[2] = m1[3 * s + 2] / v;
    }
    int64_t o = (int64_t)perm[s] * 3;
    if (wrap_abs) {
        Pos4 y = pos[s];
        double L[3] = {Lx, Ly, Lz};
        double q[3] = {y.x + c[0], y.y + c[1], y.z + c[2]};
        for (int a = 0; a < 3; a++) {
            double t = fmod(q[a], L[a]);
            if (t < 0) t += L[a];
            if (t >= L[a]) t -= L[a];
            out[o + a] = t;
        }
    } else {
        out[o] = -c[0];
        out[o + 1] = -c[1];
        out[o + 2] = -c[2];
    }
}

__global__ void status_kernel(const uint8_t* __restrict__ st, const int32_t* __restrict__ perm,
                              int64_t N, uint8_t* __restrict__ out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < N) out[perm[s]] = st[s];
}

int status_to_user(const DeviceState& d, uint8_t* out, cudaStream_t s) {
    status_kernel<<<(unsigned)((d.N + 255) / 256), 256, 0, s>>>(d.status, d.perm, d.N, out);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

int centroids_user(const DeviceState& d, double* out, int wrap_abs, cudaStream_t s) {
    centroid_kernel<<<(unsigned)((d.N + 255) / 256), 256, 0, s>>>(
        d.pos, d.m1, d.vol, d.perm, d.N, d.L[0], d.L[1], d.L[2], wrap_abs, out);
        note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

__global__ void mass_kernel(const double* __restrict__ nu, int64_t N, double* __restrict__ part) {
    __shared__ double sh[32];
    double t = 0, mn = INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = nu[i];
        t += v;
        mn = fmin(mn, isfinite(v) ? v : -INFINITY);
    }
    double a = block_sum(t, sh);
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(FULLMASK, mn, o));
    __shared__ double mm[32];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) mm[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = INFINITY;
        for (int u = 0; u < (int)(blockDim.x >> 5); u++) m = fmin(m, mm[u]);
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = m;
    }
}

__global__ void nonfinite_kernel(const double* __restrict__ v, int64_t n,
                                 int32_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) *flag = 1;  // every writer stores the same value
}

// *ok = every v[i], i < n (device memory), is finite; synchronises s
int all_finite(DeviceState& d, const double* v, int64_t n, bool* ok, cudaStream_t s) {
    int32_t* flag = d.counters + 24;
    SDOT_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    int64_t nb = (n + 255) / 256;
    if (nb > 8 * num_sms()) nb = 8 * num_sms();
    if (nb < 1) nb = 1;
    nonfinite_kernel<<<(unsigned)nb, 256, 0, s>>>(v, n, flag);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    int32_t h = 0;
    SDOT_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    *ok = h == 0;
    return SDOT_OK;
}

int check_masses(const DeviceState& d, double* sum_out, double* min_out, cudaStream_t s) {
    const int nb = 64;
    mass_kernel<<<nb, 256, 0, s>>>(d.nu, d.N, d.partials);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    double h[2 * nb];
    SDOT_CUDA_TRY(cudaMemcpyAsync(h, d.partials, sizeof h, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    double t = 0, m = INFINITY;
    for (int b = 0; b < nb; b++) {
        t += h[2 * b];
        m = fmin(m, h[2 * b + 1]);
    }
    *sum_out = t;
    *min_out = m;
    return SDOT_OK;
}

}  // namespace sdot
