// Laguerre cell clipping: volumes, first moments and facet areas of every cell, in up
// to three passes per evaluation (the per-cell work is in cell.cuh):
//   pass 1  every cell: clipped by its first candidates (its facets in the previous
//           diagram, else its k nearest seeds) and certified by the security walk;
//           a cell with a possible unseen cutter is re-queued;
//   pass 2  the re-queued cells: the walk clips every seed that cuts;
//   pass 3  FP64 re-clip, with the large polytope capacity, of the cells that failed
//           the FP32 consistency check or overflowed the small capacity.
#include <float.h>
#include <math.h>

#include <string>
#include <vector>

#include "cell.cuh"

namespace sdot {

constexpr int WARPS_PER_BLOCK_CLIP = 4;

// resident blocks per SM a polytope size allows (shared memory), at most 8
template <typename R, class C>
constexpr int clip_min_blocks() {
    return (int)((227u * 1024u) / (WARPS_PER_BLOCK_CLIP * sizeof(Poly<R, C>))) < 8
               ? (int)((227u * 1024u) / (WARPS_PER_BLOCK_CLIP * sizeof(Poly<R, C>)))
               : 8;
}

template <typename R, class C, int MODE>
__global__ void __launch_bounds__(WARPS_PER_BLOCK_CLIP * 32, (clip_min_blocks<R, C>()))
    clip_kernel(const __grid_constant__ ClipParams cp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Poly<R, C>* polys = reinterpret_cast<Poly<R, C>*>(smem_raw);
    const int lane = threadIdx.x & 31;
    Poly<R, C>& P = polys[threadIdx.x >> 5];
    const float psimax_glob = top_psimax(cp, lane);
    const float halfLmin = 0.5f * fminf(cp.Lt[0], fminf(cp.Lt[1], cp.Lt[2]));
    int carried = 0;  // cells certified by a carried certificate
    while (true) {
        int64_t w = 0;
        if (lane == 0) w = atomicAdd(cp.work_counter, 1);
        w = __shfl_sync(FULLMASK, w, 0);
        if (w >= cp.nwork) break;
        carried += process_cell<R, C, MODE>(P, cp, w, psimax_glob, halfLmin, lane) ? 1 : 0;
    }
    if (lane == 0 && carried) atomicAdd(cp.cert_carried, carried);
}

// The same pass over the work items of several contexts in one persistent launch (a
// batch of server jobs): item w of the batch belongs to the job j with
// start[j] <= w < start[j + 1] and is that job's item w - start[j].
struct ClipBatch {
    const ClipParams* jobs;       // njobs entries, device memory
    const int64_t* start;         // njobs + 1 prefix sums of the jobs' nwork
    unsigned long long* counter;  // next batch item
    int njobs;
};

template <typename R, class C, int MODE>
__global__ void __launch_bounds__(WARPS_PER_BLOCK_CLIP * 32, (clip_min_blocks<R, C>()))
    clip_batch_kernel(ClipBatch bt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Poly<R, C>* polys = reinterpret_cast<Poly<R, C>*>(smem_raw);
    const int lane = threadIdx.x & 31;
    Poly<R, C>& P = polys[threadIdx.x >> 5];
    const long long total = bt.start[bt.njobs];
    while (true) {
        long long w = 0;
        if (lane == 0) w = (long long)atomicAdd(bt.counter, 1ull);
        w = __shfl_sync(FULLMASK, w, 0);
        if (w >= total) break;
        // the last job j with start[j] <= w (jobs without items are skipped)
        int lo = 0, hi = bt.njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bt.start[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const ClipParams& cp = bt.jobs[lo];
        const float psimax_glob = top_psimax(cp, lane);
        const float halfLmin = 0.5f * fminf(cp.Lt[0], fminf(cp.Lt[1], cp.Lt[2]));
        process_cell<R, C, MODE>(P, cp, (int64_t)(w - bt.start[lo]), psimax_glob, halfLmin,
                                 lane);
    }
}

// ---------------------------------------------------------------------------
// per-evaluation preparation: normalised float positions and the psi pyramid
// ---------------------------------------------------------------------------
__global__ void posf_kernel(const Pos4* __restrict__ pos, const double* __restrict__ psi,
                            int64_t N, double inv_a, double inv_a2, double hx, double hy,
                            double hz, int Gx, int Gy, int Gz, float4* __restrict__ posf,
                            float* __restrict__ pslo, int32_t* __restrict__ leafc,
                            uint4* __restrict__ ioff) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    Pos4 y = pos[s];
    double h[3] = {hx, hy, hz};
    int G[3] = {Gx, Gy, Gz};
    double p[3] = {y.x, y.y, y.z};
    int c[3];
    float off[3];
    uint32_t io[3];
    for (int a = 0; a < 3; a++) {
        int cc = (int)floor(p[a] / h[a]);
        cc = cc < 0 ? 0 : (cc >= G[a] ? G[a] - 1 : cc);
        c[a] = cc;
        double f = p[a] - cc * h[a];
        off[a] = (float)(f * inv_a);
        double fx = floor(f / h[a] * 4294967296.0);
        fx = fx < 0.0 ? 0.0 : (fx > 4294967295.0 ? 4294967295.0 : fx);
        io[a] = (uint32_t)fx;
    }
    double q = psi[s] * inv_a2;
    float hi = (float)q;
    posf[s] = make_float4(off[0], off[1], off[2], hi);
    pslo[s] = (float)(q - (double)hi);
    leafc[s] = c[0] | (c[1] << 10) | (c[2] << 20);
    ioff[s] = make_uint4(io[0], io[1], io[2], 0u);
}

__global__ void leaf_max_kernel(const int32_t* __restrict__ cell_start, int64_t ncell,
                                const double* __restrict__ psi, double inv_a2,
                                float* __restrict__ out) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int32_t b = cell_start[c], e = cell_start[c + 1];
    double m = -INFINITY;
    for (int32_t s = b; s < e; s++) m = fmax(m, psi[s]);
    out[c] = (b == e) ? -INFINITY : __double2float_ru(m * inv_a2 * (1.0 + 1e-15 * (m > 0 ? 1 : -1)));
}

__global__ void level_max_kernel(const float* __restrict__ in, int dx, int dy, int dz,
                                 float* __restrict__ out, int ox, int oy, int oz) {
    int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (int64_t)ox * oy * oz) return;
    int X = (int)(n % ox), Y = (int)((n / ox) % oy), Z = (int)(n / ((int64_t)ox * oy));
    float m = -INFINITY;
    for (int c = 0; c < 64; c++) {
        int x = 4 * X + (c & 3), y = 4 * Y + ((c >> 2) & 3), z = 4 * Z + (c >> 4);
        if (x < dx && y < dy && z < dz) m = fmaxf(m, in[((int64_t)z * dy + y) * dx + x]);
    }
    out[n] = m;
}

// Change of psi since the previous evaluation of the context: the largest and smallest
// psi - psi_prev in units of a^2 (rounded outward, as order-preserving integers for the
// atomics: mm[0] the maximum, mm[1] the minimum); psi_prev then takes psi. Only
// differences of psi shape the diagram, so a carried certificate consumes max - min.
__global__ void psi_change_kernel(const double* __restrict__ psi, double* __restrict__ prev,
                                  int64_t N, double inv_a2, uint32_t* __restrict__ mm) {
    float hi = -INFINITY, lo = INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double p = psi[i];
        const double dv = (p - prev[i]) * inv_a2;
        hi = fmaxf(hi, __double2float_ru(dv));
        lo = fminf(lo, __double2float_rd(dv));
        prev[i] = p;
    }
    uint32_t h = f2ord(hi), l = f2ord(lo);
    h = __reduce_max_sync(FULLMASK, h);
    l = __reduce_min_sync(FULLMASK, l);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&mm[0], h);
        atomicMin(&mm[1], l);
    }
}

int build_pyramid(DeviceState& d, const double* psi, cudaStream_t s) {
    const int64_t N = d.N;
    uint32_t* mm = reinterpret_cast<uint32_t*>(d.counters + 30);
    SDOT_CUDA_TRY(cudaMemsetAsync(mm, 0, 4, s));
    SDOT_CUDA_TRY(cudaMemsetAsync(mm + 1, 0xff, 4, s));
    psi_change_kernel<<<2 * num_sms(), 256, 0, s>>>(psi, d.psi_prev, N, 1.0 / (d.a * d.a), mm);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    posf_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
        d.pos, psi, N, 1.0 / d.a, 1.0 / (d.a * d.a), d.grid.h[0], d.grid.h[1], d.grid.h[2],
        d.grid.G[0], d.grid.G[1], d.grid.G[2], d.posf, d.pslo, d.leafc, d.ioff);
        note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    Pyramid& P = d.pyr;
    leaf_max_kernel<<<(unsigned)((d.grid.ncell + 255) / 256), 256, 0, s>>>(
        d.grid.cell_start, d.grid.ncell, psi, 1.0 / (d.a * d.a), P.psimax + P.off[0]);
        note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    for (int l = 1; l < P.nlev; l++) {
        int64_t n = (int64_t)P.dim[l][0] * P.dim[l][1] * P.dim[l][2];
        level_max_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
            P.psimax + P.off[l - 1], P.dim[l - 1][0], P.dim[l - 1][1], P.dim[l - 1][2],
            P.psimax + P.off[l], P.dim[l][0], P.dim[l][1], P.dim[l][2]);
            note_launch();
        SDOT_CUDA_TRY(cudaGetLastError());
    }
    return SDOT_OK;
}

// ---------------------------------------------------------------------------
// reductions over the cells
// ---------------------------------------------------------------------------
constexpr int RED_BLOCKS = 256;

__global__ void cell_reduce_kernel(const double* __restrict__ vol, const double* __restrict__ nu,
                                   const uint8_t* __restrict__ status, int64_t N,
                                   double* __restrict__ part) {
    double sv = 0, mr = 0, l2 = 0, mv = INFINITY, ne = 0;
    uint32_t fl = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = vol[i], g = nu[i] - v;
        sv += v;
        mr = fmax(mr, fabs(g) / nu[i]);
        l2 += g * g;
        mv = fmin(mv, v);
        if (!(v > 0)) ne += 1;
        fl |= status[i];
    }
    __shared__ double sh[6][8];
    for (int o = 16; o > 0; o >>= 1) {
        sv += __shfl_xor_sync(FULLMASK, sv, o);
        mr = fmax(mr, __shfl_xor_sync(FULLMASK, mr, o));
        l2 += __shfl_xor_sync(FULLMASK, l2, o);
        mv = fmin(mv, __shfl_xor_sync(FULLMASK, mv, o));
        ne += __shfl_xor_sync(FULLMASK, ne, o);
        fl |= __shfl_xor_sync(FULLMASK, fl, o);
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = sv;
        sh[1][w] = mr;
        sh[2][w] = l2;
        sh[3][w] = mv;
        sh[4][w] = ne;
        sh[5][w] = (double)fl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int u = 1; u < (int)(blockDim.x >> 5); u++) {
            sh[0][0] += sh[0][u];
            sh[1][0] = fmax(sh[1][0], sh[1][u]);
            sh[2][0] += sh[2][u];
            sh[3][0] = fmin(sh[3][0], sh[3][u]);
            sh[4][0] += sh[4][u];
            sh[5][0] = (double)((uint32_t)sh[5][0] | (uint32_t)sh[5][u]);
        }
        for (int q = 0; q < 6; q++) part[blockIdx.x * 6 + q] = sh[q][0];
    }
}

__global__ void cell_reduce_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    double sv = 0, mr = 0, l2 = 0, mv = INFINITY, ne = 0;
    uint32_t fl = 0;
    for (int b = 0; b < nb; b++) {
        sv += part[b * 6];
        mr = fmax(mr, part[b * 6 + 1]);
        l2 += part[b * 6 + 2];
        mv = fmin(mv, part[b * 6 + 3]);
        ne += part[b * 6 + 4];
        fl |= (uint32_t)part[b * 6 + 5];
    }
    out[0] = sv;
    out[1] = mr;
    out[2] = sqrt(l2);
    out[3] = mv;
    out[4] = ne;
    out[5] = (double)fl;
}

// Setup of a persistent clipping kernel, once per instantiation: blocks per SM from the
// occupancy at the largest shared-memory carveout, then the smallest carveout that still
// holds that many blocks, so the rest of the SM's memory stays L1 (which caches the
// lanes' local memory). The occupancy is checked again at that carveout and the largest
// one restored if it dropped.
template <typename K>
static cudaError_t clip_setup(K kernel, size_t smem, int* blocks) {
    const int threads = WARPS_PER_BLOCK_CLIP * 32;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int dev = 0, smem_sm = 0, resv = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) ==
            cudaSuccess &&
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) ==
            cudaSuccess &&
        smem_sm > 0) {
        // shared memory is allocated per block in 128-byte units, plus the reserved part;
        // the percentage is rounded down and the driver rounds it up to a supported size
        const size_t per_block = (smem + (size_t)resv + 127) / 128 * 128;
        const int pct = (int)((size_t)per_sm * per_block * 100 / (size_t)smem_sm);
        if (pct < 100 &&
            cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct) ==
                cudaSuccess) {
            int again = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&again, kernel, threads, smem) !=
                    cudaSuccess ||
                again < per_sm)
                cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        }
        cudaGetLastError();
    }
    *blocks = per_sm * num_sms();
    return cudaSuccess;
}

template <typename R, class C, int MODE>
static int launch_clip(const ClipParams& cp, cudaStream_t s) {
    const size_t smem = sizeof(Poly<R, C>) * WARPS_PER_BLOCK_CLIP;
    // kernel attributes and the persistent grid size, set once per instantiation
    // (thread-safe: contexts of different host threads launch concurrently)
    struct Setup {
        int blocks;
        cudaError_t err;
    };
    static const Setup setup = [smem] {
        Setup u{0, cudaSuccess};
        u.err = clip_setup(clip_kernel<R, C, MODE>, smem, &u.blocks);
        return u;
    }();
    if (setup.err != cudaSuccess) {
        set_error(std::string("clip kernel setup: ") + cudaGetErrorString(setup.err));
        return SDOT_ERR_CUDA;
    }
    const int blocks = setup.blocks;
    int64_t need = (cp.nwork + WARPS_PER_BLOCK_CLIP - 1) / WARPS_PER_BLOCK_CLIP;
    int nb = (int)(need < blocks ? need : blocks);
    if (nb < 1) return SDOT_OK;
    clip_kernel<R, C, MODE><<<nb, WARPS_PER_BLOCK_CLIP * 32, smem, s>>>(cp);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

// clipping parameters of one evaluation of context d at psi (no work counter,
// work list or counters yet)
static ClipParams make_clip_params(DeviceState& d, const double* psi) {
    ClipParams cp;
    cp.N = d.N;
    cp.k = d.k;
    cp.a = d.a;
    cp.inv_a = 1.0 / d.a;
    cp.inv_a2 = 1.0 / (d.a * d.a);
    for (int a = 0; a < 3; a++) {
        cp.L[a] = d.L[a];
        cp.halfL[a] = 0.5 * d.L[a];
        cp.Lt[a] = (float)(d.L[a] / d.a);
        cp.halfLt[a] = 0.5f * cp.Lt[a];
        cp.ht[a] = (float)(d.grid.h[a] / d.a);
        cp.G[a] = d.grid.G[a];
    }
    cp.pos = d.pos;
    cp.posf = d.posf;
    cp.pslo = d.pslo;
    cp.ioff = d.ioff;
    for (int a = 0; a < 3; a++) cp.hfix[a] = (float)(d.grid.h[a] / d.a / 4294967296.0);
    cp.leafc = d.leafc;
    cp.facets_valid = d.facets_valid;
    cp.psi = psi;
    cp.knn = d.knn;
    cp.knn_d2k = d.knn_d2k;
    cp.cell_start = d.grid.cell_start;
    cp.pyr = d.pyr;
    for (int l = 0; l < MAXLEV; l++)
        for (int a = 0; a < 3; a++) cp.nsz[l][a] = (float)((double)(1 << (2 * l)) * d.grid.h[a] / d.a);
    cp.vol = d.vol;
    cp.m1 = d.m1;
    cp.anchor = d.anchor;
    cp.status = d.status;
    cp.fcnt = d.fcnt;
    cp.fcol = d.fcol;
    cp.fval = d.fval;
    cp.topo = d.topo;
    cp.topo_n = d.topo_n;
    cp.cert_f = d.cert_f;
    cp.cert_s = d.cert_s;
    cp.cert_j = d.cert_j;
    cp.cert_n = d.cert_n;
    cp.cert_dpsi = reinterpret_cast<const uint32_t*>(d.counters + 30);
    cp.cert_carried = d.counters + 29;
    cp.cert_use = d.carry;
    cp.queue_out = d.queue;
    cp.queue_cnt = d.counters + 0;
    cp.q64_out = d.queue64;
    cp.q64_cnt = d.counters + 1;
    cp.counters64 = (unsigned long long*)(d.counters + 8);
    cp.work_counter = nullptr;
    cp.worklist = nullptr;
    cp.nwork = d.N;
    cp.pass = 1;
    return cp;
}

// the cells of context d at its current psi, for rebuilding them from their facets in
// FP64 (mesh.cu)
ClipParams mesh_clip_params(DeviceState& d) { return make_clip_params(d, d.psi); }

int evaluate_cells(DeviceState& d, const double* psi, int precision, EvalResult* res,
                   cudaStream_t s) {
    NvtxRange nv("laguerre_cells");
    int rc = build_pyramid(d, psi, s);
    if (rc) return rc;
    ClipParams cp = make_clip_params(d, psi);
    SDOT_CUDA_TRY(cudaMemsetAsync(d.counters, 0, 8 * sizeof(int32_t), s));
    SDOT_CUDA_TRY(cudaMemsetAsync(d.counters + 29, 0, sizeof(int32_t), s));

    cudaEvent_t e0, e1, ep1, ep2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&ep1);
    cudaEventCreate(&ep2);
    cp.counters64 = (unsigned long long*)(d.counters + 8);
    SDOT_CUDA_TRY(cudaMemsetAsync(d.counters + 8, 0, 64, s));
    cudaEventRecord(e0, s);
    // pass 1: every cell, kNN planes + security test
    cp.work_counter = d.counters + 2;
    cp.worklist = nullptr;
    cp.nwork = d.N;
    cp.pass = 1;
    rc = precision == SDOT_PREC_FP64 ? launch_clip<double, CapS, MODE_CERTIFY>(cp, s)
                                     : launch_clip<float, CapS, MODE_CERTIFY>(cp, s);
    if (rc) return rc;
    cudaEventRecord(ep1, s);
    int32_t cnt[2];
    SDOT_CUDA_TRY(cudaMemcpyAsync(cnt, d.counters, 8, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t requeued = cnt[0];
    // pass 2: re-queued cells, full walk with clipping
    if (requeued > 0) {
        cp.work_counter = d.counters + 4;
        cp.worklist = d.queue;
        cp.nwork = requeued;
        cp.pass = 2;
        rc = precision == SDOT_PREC_FP64 ? launch_clip<double, CapS, MODE_FULL>(cp, s)
                                         : launch_clip<float, CapS, MODE_FULL>(cp, s);
        if (rc) return rc;
        SDOT_CUDA_TRY(cudaMemcpyAsync(cnt, d.counters, 8, cudaMemcpyDeviceToHost, s));
        SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    }
    cudaEventRecord(ep2, s);
    int64_t reclipped = cnt[1];
    // pass 3: FP64 re-clip of the cells failing the FP32 checks or over the small
    // capacity: the small polytope first (its overflows are appended to the same queue),
    // then the large one for those
    if (reclipped > 0) {
        cp.pass = 3;
        cp.work_counter = d.counters + 5;
        cp.worklist = d.queue64;
        cp.nwork = reclipped;
        if (precision != SDOT_PREC_FP64) {
            if ((rc = launch_clip<double, CapS, MODE_FULL>(cp, s))) return rc;
            SDOT_CUDA_TRY(cudaMemcpyAsync(cnt, d.counters, 8, cudaMemcpyDeviceToHost, s));
            SDOT_CUDA_TRY(cudaStreamSynchronize(s));
            cp.work_counter = d.counters + 6;
            cp.worklist = d.queue64 + reclipped;
            cp.nwork = (int64_t)cnt[1] - reclipped;
        }
        if (cp.nwork > 0 && (rc = launch_clip<double, CapL, MODE_FULL>(cp, s))) return rc;
    }
    cudaEventRecord(e1, s);
    cell_reduce_kernel<<<RED_BLOCKS, 256, 0, s>>>(d.vol, d.nu, d.status, d.N, d.partials);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    cell_reduce_final<<<1, 32, 0, s>>>(d.partials, RED_BLOCKS, d.scal);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    double h[6];
    SDOT_CUDA_TRY(cudaMemcpyAsync(h, d.scal, sizeof h, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventElapsedTime(&res->ms_pass[0], e0, ep1);
    cudaEventElapsedTime(&res->ms_pass[1], ep1, ep2);
    cudaEventElapsedTime(&res->ms_pass[2], ep2, e1);
    SDOT_CUDA_TRY(cudaMemcpy(res->work, d.counters + 8, 64, cudaMemcpyDeviceToHost));
    int32_t carried = 0;
    SDOT_CUDA_TRY(cudaMemcpy(&carried, d.counters + 29, 4, cudaMemcpyDeviceToHost));
    res->carried = carried;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(ep1);
    cudaEventDestroy(ep2);
    d.facets_valid = 1;  // every cell now holds its facets of this diagram
    res->sum_vol = h[0];
    res->max_rel_err = h[1];
    res->l2_err = h[2];
    res->min_vol = h[3];
    res->n_empty = (int64_t)h[4];
    res->flags = (uint32_t)h[5];
    res->requeued = requeued;
    res->reclipped = reclipped;
    res->ms = ms;
    return SDOT_OK;
}


// ---------------------------------------------------------------------------
// batched evaluation: one persistent launch per pass over the cells of several
// contexts (the server's jobs)
// ---------------------------------------------------------------------------
template <typename R, class C, int MODE>
static int launch_clip_batch(const ClipBatch& bt, int64_t total, cudaStream_t s) {
    const size_t smem = sizeof(Poly<R, C>) * WARPS_PER_BLOCK_CLIP;
    struct Setup {
        int blocks;
        cudaError_t err;
    };
    static const Setup setup = [smem] {
        Setup u{0, cudaSuccess};
        u.err = clip_setup(clip_batch_kernel<R, C, MODE>, smem, &u.blocks);
        return u;
    }();
    if (setup.err != cudaSuccess) {
        set_error(std::string("clip batch kernel setup: ") + cudaGetErrorString(setup.err));
        return SDOT_ERR_CUDA;
    }
    const int64_t need = (total + WARPS_PER_BLOCK_CLIP - 1) / WARPS_PER_BLOCK_CLIP;
    const int nb = (int)(need < setup.blocks ? need : setup.blocks);
    if (nb < 1) return SDOT_OK;
    clip_batch_kernel<R, C, MODE><<<nb, WARPS_PER_BLOCK_CLIP * 32, smem, s>>>(bt);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

// Job tables of a batch: one slot per launch of a pass (the FP32 and the FP64 group);
// the host copies are pinned and reused after the stream has been synchronised.
struct BatchScratch {
    int cap = 0;
    ClipParams* jobs_dev[2] = {nullptr, nullptr};
    int64_t* start_dev[2] = {nullptr, nullptr};
    unsigned long long* counter_dev = nullptr;  // one per slot
    ClipParams* jobs_host[2] = {nullptr, nullptr};
    int64_t* start_host[2] = {nullptr, nullptr};
    int32_t* cnt_host = nullptr;  // 2 per job: re-queued, FP64 re-clip counts
    double* red_host = nullptr;   // 6 per job: the reductions of cell_reduce_final
};

void batch_scratch_destroy(BatchScratch* b) {
    if (!b) return;
    for (int t = 0; t < 2; t++) {
        cudaFree(b->jobs_dev[t]);
        cudaFree(b->start_dev[t]);
        cudaFreeHost(b->jobs_host[t]);
        cudaFreeHost(b->start_host[t]);
    }
    cudaFree(b->counter_dev);
    cudaFreeHost(b->cnt_host);
    cudaFreeHost(b->red_host);
    delete b;
}

int batch_scratch_create(int cap, BatchScratch** out) {
    *out = nullptr;
    if (cap < 1) return SDOT_ERR_ARG;
    BatchScratch* b = new BatchScratch();
    b->cap = cap;
    bool ok = true;
    for (int t = 0; t < 2 && ok; t++) {
        ok = cudaMalloc(&b->jobs_dev[t], sizeof(ClipParams) * cap) == cudaSuccess &&
             cudaMalloc(&b->start_dev[t], sizeof(int64_t) * (cap + 1)) == cudaSuccess &&
             cudaMallocHost(&b->jobs_host[t], sizeof(ClipParams) * cap) == cudaSuccess &&
             cudaMallocHost(&b->start_host[t], sizeof(int64_t) * (cap + 1)) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&b->counter_dev, sizeof(unsigned long long) * 2) == cudaSuccess &&
         cudaMallocHost(&b->cnt_host, sizeof(int32_t) * 2 * cap) == cudaSuccess &&
         cudaMallocHost(&b->red_host, sizeof(double) * 6 * cap) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        batch_scratch_destroy(b);
        set_error("batch scratch: allocation failed");
        return SDOT_ERR_OOM;
    }
    *out = b;
    return SDOT_OK;
}

// one launch of pass MODE in precision R over the work items nwork[j] of the jobs with
// take[j] (items: worklist of cps[j], or cells 0..nwork[j]-1)
template <typename R, class C, int MODE>
static int launch_table(const std::vector<ClipParams>& cps, const std::vector<int64_t>& nwork,
                        const std::vector<char>& take, int slot, BatchScratch* sc,
                        cudaStream_t s) {
    int m = 0;
    int64_t total = 0;
    ClipParams* hj = sc->jobs_host[slot];
    int64_t* hs = sc->start_host[slot];
    for (size_t j = 0; j < cps.size(); j++) {
        if (!take[j] || nwork[j] <= 0) continue;
        hj[m] = cps[j];
        hj[m].nwork = nwork[j];
        hj[m].work_counter = nullptr;  // the batch counter hands out the items
        hs[m] = total;
        total += nwork[j];
        m++;
    }
    if (m == 0) return SDOT_OK;
    hs[m] = total;
    SDOT_CUDA_TRY(cudaMemcpyAsync(sc->jobs_dev[slot], hj, sizeof(ClipParams) * m,
                                  cudaMemcpyHostToDevice, s));
    SDOT_CUDA_TRY(cudaMemcpyAsync(sc->start_dev[slot], hs, sizeof(int64_t) * (m + 1),
                                  cudaMemcpyHostToDevice, s));
    SDOT_CUDA_TRY(cudaMemsetAsync(sc->counter_dev + slot, 0, sizeof(unsigned long long), s));
    ClipBatch bt;
    bt.jobs = sc->jobs_dev[slot];
    bt.start = sc->start_dev[slot];
    bt.counter = sc->counter_dev + slot;
    bt.njobs = m;
    return launch_clip_batch<R, C, MODE>(bt, total, s);
}

// the per-job counters (re-queued, FP64 re-clip) of every job, after a sync of s
static int read_counts(DeviceState* const* ds, int n, BatchScratch* sc, cudaStream_t s) {
    for (int j = 0; j < n; j++)
        SDOT_CUDA_TRY(cudaMemcpyAsync(sc->cnt_host + 2 * j, ds[j]->counters, 2 * sizeof(int32_t),
                                      cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    return SDOT_OK;
}

int evaluate_cells_batch(DeviceState* const* ds, const double* const* psis, const int* precs,
                         EvalResult* res, int n, BatchScratch* sc, cudaStream_t s) {
    if (n < 1 || !sc || n > sc->cap) {
        set_error("evaluate_cells_batch: batch size out of range");
        return SDOT_ERR_ARG;
    }
    int rc;
    std::vector<ClipParams> cps((size_t)n);
    std::vector<int64_t> nwork((size_t)n);
    std::vector<char> is64((size_t)n), is32((size_t)n), all((size_t)n, 1);
    for (int j = 0; j < n; j++) {
        DeviceState& d = *ds[j];
        if ((rc = build_pyramid(d, psis[j], s))) return rc;
        cps[j] = make_clip_params(d, psis[j]);
        SDOT_CUDA_TRY(cudaMemsetAsync(d.counters, 0, 8 * sizeof(int32_t), s));
        SDOT_CUDA_TRY(cudaMemsetAsync(d.counters + 8, 0, 64, s));
        is64[j] = precs[j] == SDOT_PREC_FP64;
        is32[j] = !is64[j];
    }
    cudaEvent_t e0, e1, ep1, ep2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&ep1);
    cudaEventCreate(&ep2);
    auto cleanup = [&] {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(ep1);
        cudaEventDestroy(ep2);
    };
    cudaEventRecord(e0, s);
    // pass 1: every cell of every job
    for (int j = 0; j < n; j++) {
        cps[j].worklist = nullptr;
        cps[j].pass = 1;
        nwork[j] = ds[j]->N;
    }
    if ((rc = launch_table<float, CapS, MODE_CERTIFY>(cps, nwork, is32, 0, sc, s)) ||
        (rc = launch_table<double, CapS, MODE_CERTIFY>(cps, nwork, is64, 1, sc, s))) {
        cleanup();
        return rc;
    }
    cudaEventRecord(ep1, s);
    if ((rc = read_counts(ds, n, sc, s))) {
        cleanup();
        return rc;
    }
    std::vector<int64_t> requeued((size_t)n), reclipped((size_t)n);
    bool any = false;
    for (int j = 0; j < n; j++) {
        requeued[j] = sc->cnt_host[2 * j];
        cps[j].worklist = ds[j]->queue;
        cps[j].pass = 2;
        nwork[j] = requeued[j];
        any = any || requeued[j] > 0;
    }
    // pass 2: the re-queued cells, full walk with clipping
    if (any) {
        if ((rc = launch_table<float, CapS, MODE_FULL>(cps, nwork, is32, 0, sc, s)) ||
            (rc = launch_table<double, CapS, MODE_FULL>(cps, nwork, is64, 1, sc, s))) {
            cleanup();
            return rc;
        }
    }
    cudaEventRecord(ep2, s);
    if ((rc = read_counts(ds, n, sc, s))) {
        cleanup();
        return rc;
    }
    any = false;
    for (int j = 0; j < n; j++) {
        reclipped[j] = sc->cnt_host[2 * j + 1];
        cps[j].worklist = ds[j]->queue64;
        cps[j].pass = 3;
        nwork[j] = reclipped[j];
        any = any || nwork[j] > 0;
    }
    // pass 3: FP64 re-clip with the large capacity (FP32 cells failing the checks,
    // cells over the small capacity)
    if (any && (rc = launch_table<double, CapL, MODE_FULL>(cps, nwork, all, 0, sc, s))) {
        cleanup();
        return rc;
    }
    cudaEventRecord(e1, s);
    std::vector<unsigned long long> work((size_t)n * 8);
    for (int j = 0; j < n; j++) {
        DeviceState& d = *ds[j];
        SDOT_CUDA_TRY(cudaMemcpyAsync(work.data() + 8 * j, d.counters + 8, 64,
                                      cudaMemcpyDeviceToHost, s));
        cell_reduce_kernel<<<RED_BLOCKS, 256, 0, s>>>(d.vol, d.nu, d.status, d.N, d.partials);
        note_launch();
        SDOT_CUDA_TRY(cudaGetLastError());
        cell_reduce_final<<<1, 32, 0, s>>>(d.partials, RED_BLOCKS, d.scal);
        note_launch();
        SDOT_CUDA_TRY(cudaGetLastError());
        SDOT_CUDA_TRY(cudaMemcpyAsync(sc->red_host + 6 * j, d.scal, 6 * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    }
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0, mp[3] = {0, 0, 0};
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventElapsedTime(&mp[0], e0, ep1);
    cudaEventElapsedTime(&mp[1], ep1, ep2);
    cudaEventElapsedTime(&mp[2], ep2, e1);
    cleanup();
    for (int j = 0; j < n; j++) {
        DeviceState& d = *ds[j];
        EvalResult& r = res[j];
        const double* h = sc->red_host + 6 * j;
        for (int q = 0; q < 8; q++) r.work[q] = work[8 * j + q];
        d.facets_valid = 1;
        r.sum_vol = h[0];
        r.max_rel_err = h[1];
        r.l2_err = h[2];
        r.min_vol = h[3];
        r.n_empty = (int64_t)h[4];
        r.flags = (uint32_t)h[5];
        r.requeued = requeued[j];
        r.reclipped = reclipped[j];
        r.ms = ms;
        for (int q = 0; q < 3; q++) r.ms_pass[q] = mp[q];
    }
    return SDOT_OK;
}

}  // namespace sdot
