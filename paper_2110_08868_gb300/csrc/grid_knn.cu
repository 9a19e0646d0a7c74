// Spatial hash of the seeds and the periodic k-nearest-neighbour lists.
//
// The seeds are binned into a G^3 grid of cells of ~seeds_per_leaf seeds, sorted by
// cell (counting sort; ties inside a cell by caller index, so the order is
// deterministic) and kept in that order on the device for every later kernel.
// Each query walks rings of grid cells until its k-th distance is below the distance
// to the first unvisited ring. The distance key is (d^2, caller index) with
// d^2 = (dx*dx + dy*dy) + dz*dz of the minimum-image difference, evaluated with
// explicit round-to-nearest products and sums (no FMA) so that it is bit-identical
// to a plain IEEE binary64 evaluation.
//
// The paper computes the Laguerre diagram exactly (Sec. "Monge-Ampere-Kantorovich
// Reconstruction", eq. laguerrecell) without saying how neighbours are found; the
// kNN list is the first candidate set of the clipping kernel.
#include <float.h>
#include <limits.h>

#include "internal.cuh"

namespace sdot {

static unsigned long long g_launches = 0;
void note_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

// SM count of the device current at the first call (initialised once, thread-safe)
int num_sms() {
    static const int n = [] {
        int dev = 0, m = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
        return m > 0 ? m : 1;
    }();
    return n;
}

// ---------------------------------------------------------------------------
// exclusive scan (three-phase, recursive over block sums)
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int64_t SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T* total) {
    __shared__ T ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        T s = (lane < nw) ? ws[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    T pre = (w > 0) ? ws[w - 1] : T(0);
    *total = ws[nw - 1];
    __syncthreads();
    return pre + x - v;
}

template <typename Tin, typename Tout>
__global__ void scan_sums_kernel(const Tin* in, int64_t n, Tout* sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout t = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++)
        if (base + k < n) t += (Tout)in[base + k];
    __shared__ Tout red[32];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        Tout s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : Tout(0);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = s;
    }
}

template <typename Tin, typename Tout>
__global__ void scan_apply_kernel(const Tin* in, Tout* out, int64_t n, const Tout* offsets) {
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout v[SCAN_ITEMS];
    Tout t = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = (base + k < n) ? (Tout)in[base + k] : Tout(0);
        t += v[k];
    }
    Tout total;
    Tout pre = block_exclusive_scan<Tout>(t, &total);
    if (offsets) pre += offsets[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        if (base + k < n) out[base + k] = pre;
        pre += v[k];
    }
}

size_t scan_temp_bytes(int64_t n) {
    size_t b = 0;
    while (n > SCAN_CHUNK) {
        n = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
        b += (size_t)n * sizeof(int64_t) + 256;
    }
    return b + 256;
}

template <typename Tin, typename Tout>
static int scan_impl(const Tin* in, Tout* out, int64_t n, char* temp, cudaStream_t s) {
    if (n <= 0) return SDOT_OK;
    int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nb == 1) {
        scan_apply_kernel<Tin, Tout><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
        note_launch();
        SDOT_CUDA_TRY(cudaGetLastError());
        return SDOT_OK;
    }
    Tout* sums = reinterpret_cast<Tout*>(temp);
    char* next = temp + ((nb * sizeof(Tout) + 255) / 256) * 256;
    scan_sums_kernel<Tin, Tout><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    int rc = scan_impl<Tout, Tout>(sums, sums, nb, next, s);
    if (rc) return rc;
    scan_apply_kernel<Tin, Tout><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

int scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* temp,
                              cudaStream_t s) {
    return scan_impl<int32_t, int64_t>(in, out, n, (char*)temp, s);
}
int scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, void* temp,
                       cudaStream_t s) {
    return scan_impl<int32_t, int32_t>(in, out, n, (char*)temp, s);
}

// ---------------------------------------------------------------------------
// grid build
// ---------------------------------------------------------------------------
struct GridParams {
    int G[3];
    double h[3];
    double L[3];
};

__device__ __forceinline__ int cell_coord(double x, double h, int G) {
    int c = (int)floor(x / h);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
}

__global__ void keys_kernel(const double* __restrict__ pos, int64_t N, GridParams gp,
                            int32_t* __restrict__ key, int32_t* __restrict__ count,
                            int* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    bool ok = isfinite(x) && isfinite(y) && isfinite(z) && x >= 0.0 && y >= 0.0 &&
              z >= 0.0 && x < gp.L[0] && y < gp.L[1] && z < gp.L[2];
    if (!ok) {
        atomicOr(bad, 1);
        x = y = z = 0.0;
    }
    int cx = cell_coord(x, gp.h[0], gp.G[0]);
    int cy = cell_coord(y, gp.h[1], gp.G[1]);
    int cz = cell_coord(z, gp.h[2], gp.G[2]);
    int32_t k = (cz * gp.G[1] + cy) * gp.G[0] + cx;
    key[i] = k;
    atomicAdd(&count[k], 1);
}

__global__ void scatter_kernel(const int32_t* __restrict__ key, int64_t N,
                               const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                               int32_t* __restrict__ perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int32_t k = key[i];
    int32_t slot = start[k] + atomicAdd(&fill[k], 1);
    perm[slot] = (int32_t)i;
}

// insertion sort of each cell's seeds by caller index (cells hold few seeds)
__global__ void sort_cells_kernel(const int32_t* __restrict__ start, int64_t ncell,
                                  int32_t* __restrict__ perm) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int32_t b = start[c], e = start[c + 1];
    for (int32_t t = b + 1; t < e; t++) {
        int32_t v = perm[t];
        int32_t u = t - 1;
        while (u >= b && perm[u] > v) {
            perm[u + 1] = perm[u];
            u--;
        }
        perm[u + 1] = v;
    }
}

__global__ void finalize_sort_kernel(const double* __restrict__ pos_user, int64_t N,
                                     const int32_t* __restrict__ perm,
                                     int32_t* __restrict__ iperm, Pos4* __restrict__ pos) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    int32_t i = perm[s];
    iperm[i] = (int32_t)s;
    pos[s] = Pos4::make(pos_user[3 * (int64_t)i], pos_user[3 * (int64_t)i + 1],
                          pos_user[3 * (int64_t)i + 2], (double)i);
}

int build_grid(DeviceState& d, const double* pos_user_dev, double seeds_per_leaf, void* temp,
               cudaStream_t s, const char* who) {
    const int64_t N = d.N;
    double vol = d.L[0] * d.L[1] * d.L[2];
    double h = cbrt(seeds_per_leaf * vol / (double)N);
    GridParams gp;
    int64_t ncell = 1;
    for (int a = 0; a < 3; a++) {
        double g = floor(d.L[a] / h);
        if (g < 1) g = 1;
        if (g > 1024) g = 1024;
        gp.G[a] = (int)g;
        gp.h[a] = d.L[a] / g;
        gp.L[a] = d.L[a];
        d.grid.G[a] = gp.G[a];
        d.grid.h[a] = gp.h[a];
        ncell *= gp.G[a];
    }
    d.grid.ncell = ncell;
    // temp layout: key[N] | count[ncell] | fill[ncell] | bad | scan temp
    char* t = (char*)temp;
    int32_t* key = (int32_t*)t;
    t += ((N * 4 + 255) / 256) * 256;
    int32_t* count = (int32_t*)t;
    t += ((ncell * 4 + 255) / 256) * 256;
    int32_t* fill = (int32_t*)t;
    t += ((ncell * 4 + 255) / 256) * 256;
    int* bad = (int*)t;
    t += 256;
    SDOT_CUDA_TRY(cudaMemsetAsync(count, 0, ncell * 4, s));
    SDOT_CUDA_TRY(cudaMemsetAsync(fill, 0, ncell * 4, s));
    SDOT_CUDA_TRY(cudaMemsetAsync(bad, 0, 4, s));
    unsigned nb = (unsigned)((N + 255) / 256);
    keys_kernel<<<nb, 256, 0, s>>>(pos_user_dev, N, gp, key, count, bad);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    // cell_start = exclusive scan of counts, with cell_start[ncell] = N
    int rc = scan_exclusive_i32(count, d.grid.cell_start, ncell, t, s);
    if (rc) return rc;
    int32_t nN = (int32_t)N;
    SDOT_CUDA_TRY(cudaMemcpyAsync(d.grid.cell_start + ncell, &nN, 4, cudaMemcpyHostToDevice, s));
    scatter_kernel<<<nb, 256, 0, s>>>(key, N, d.grid.cell_start, fill, d.perm);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    sort_cells_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(d.grid.cell_start, ncell,
                                                                     d.perm);
                                                                     note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    finalize_sort_kernel<<<nb, 256, 0, s>>>(pos_user_dev, N, d.perm, d.iperm, d.pos);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    int hbad = 0;
    SDOT_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) {
        set_error(std::string(who) + ": a position is not finite or lies outside [0, box)");
        return SDOT_ERR_ARG;
    }
    return SDOT_OK;
}

// ---------------------------------------------------------------------------
// kNN
// ---------------------------------------------------------------------------
struct KnnParams {
    int G[3];
    double h[3];
    double L[3];
    double halfL[3];
    int64_t N;
    int k;
};

// minimum-image component, same rule as a plain statement of it:
// if dx > L/2 subtract L, else if dx < -L/2 add L
__device__ __forceinline__ double wrap_d(double dx, double L, double halfL) {
    if (dx > halfL) return __dsub_rn(dx, L);
    if (dx < -halfL) return __dadd_rn(dx, L);
    return dx;
}

__device__ __forceinline__ double dist2_exact(const Pos4& a, const Pos4& b,
                                              const KnnParams& p) {
    double dx = wrap_d(__dsub_rn(b.x, a.x), p.L[0], p.halfL[0]);
    double dy = wrap_d(__dsub_rn(b.y, a.y), p.L[1], p.halfL[1]);
    double dz = wrap_d(__dsub_rn(b.z, a.z), p.L[2], p.halfL[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

template <int K>
struct TopK {
    double d[K];
    int o[K];   // caller index (tie key)
    int s[K];   // sorted index
    __device__ void init() {
#pragma unroll
        for (int t = 0; t < K; t++) {
            d[t] = DBL_MAX;
            o[t] = INT_MAX;
            s[t] = -1;
        }
    }
    __device__ __forceinline__ static bool less(double d1, int o1, double d2, int o2) {
        return d1 < d2 || (d1 == d2 && o1 < o2);
    }
    __device__ __forceinline__ void insert(double cd, int co, int cs) {
        if (!less(cd, co, d[K - 1], o[K - 1])) return;
#pragma unroll
        for (int t = K - 1; t >= 0; t--) {
            if (less(cd, co, d[t], o[t])) {
                bool sh = (t > 0) && less(cd, co, d[t - 1], o[t - 1]);
                d[t] = sh ? d[t - 1] : cd;
                o[t] = sh ? o[t - 1] : co;
                s[t] = sh ? s[t - 1] : cs;
            }
        }
    }
};

// Exact search of query q: rings of grid cells with the FP64 key, from ring 0 until
// the k-th key is below the squared distance to the first unvisited ring (brute force
// over all seeds when the rings would wrap onto visited cells).
template <int K>
__device__ __noinline__ void knn_exact(const Pos4* __restrict__ pos,
                                       const int32_t* __restrict__ cell_start,
                                       const KnnParams& p, int64_t q, TopK<K>& top) {
    const Pos4 yi = pos[q];
    top.init();
    int c[3];
    double m = DBL_MAX;
    {
        const double xs[3] = {yi.x, yi.y, yi.z};
        for (int a = 0; a < 3; a++) {
            int cc = (int)floor(xs[a] / p.h[a]);
            cc = cc < 0 ? 0 : (cc >= p.G[a] ? p.G[a] - 1 : cc);
            c[a] = cc;
            const double f = xs[a] - cc * p.h[a];
            double ma = fmin(f, p.h[a] - f);
            if (ma < 0) ma = 0;
            m = fmin(m, ma);
        }
    }
    const int Gmin = min(p.G[0], min(p.G[1], p.G[2]));
    const int k = p.k;
    bool done = false;
    for (int r = 0; !done; r++) {
        if (2 * r + 1 > Gmin) {
            // the next ring would wrap onto visited cells: finish by brute force
            top.init();
            for (int64_t t = 0; t < p.N; t++) {
                if (t == q) continue;
                const Pos4 yj = pos[t];
                top.insert(dist2_exact(yi, yj, p), (int)yj.w, (int)t);
            }
            break;
        }
        for (int oz = -r; oz <= r; oz++) {
            const int cz = ((c[2] + oz) % p.G[2] + p.G[2]) % p.G[2];
            for (int oy = -r; oy <= r; oy++) {
                const int cy = ((c[1] + oy) % p.G[1] + p.G[1]) % p.G[1];
                const bool face = (oz == -r || oz == r || oy == -r || oy == r);
                const int step = (face || r == 0) ? 1 : 2 * r;
                for (int ox = -r; ox <= r; ox += step) {
                    const int cx = ((c[0] + ox) % p.G[0] + p.G[0]) % p.G[0];
                    const int64_t cell = ((int64_t)cz * p.G[1] + cy) * p.G[0] + cx;
                    const int32_t b = cell_start[cell], e = cell_start[cell + 1];
                    for (int32_t t = b; t < e; t++) {
                        if (t == q) continue;
                        const Pos4 yj = pos[t];
                        top.insert(dist2_exact(yi, yj, p), (int)yj.w, t);
                    }
                }
            }
        }
        // every unvisited seed lies at least r*h + m away
        double bound = DBL_MAX;
        for (int a = 0; a < 3; a++) bound = fmin(bound, r * p.h[a] + m);
        double kth = DBL_MAX;
#pragma unroll
        for (int t = 0; t < K; t++)
            if (t == k - 1) kth = top.d[t];
        if (kth < DBL_MAX && kth < bound * bound * (1.0 - 1e-12)) done = true;
    }
}

// Grid-local FP32 offsets of every seed (in units of the grid cell) and its grid cell,
// for the FP32 pass of the search.
__global__ void knn_prep_kernel(const Pos4* __restrict__ pos, int64_t N, KnnParams p,
                                float4* __restrict__ off, int32_t* __restrict__ cellc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const Pos4 y = pos[t];
    const double xs[3] = {y.x, y.y, y.z};
    int c[3];
    float o[3];
    for (int a = 0; a < 3; a++) {
        int cc = (int)floor(xs[a] / p.h[a]);
        cc = cc < 0 ? 0 : (cc >= p.G[a] ? p.G[a] - 1 : cc);
        c[a] = cc;
        o[a] = (float)((xs[a] - cc * p.h[a]) / p.h[a]);
    }
    off[t] = make_float4(o[0], o[1], o[2], 0.f);
    cellc[t] = c[0] | (c[1] << 10) | (c[2] << 20);
}

// k nearest seeds of every query. A first pass in FP32 keeps the K + 8 smallest
// approximate squared distances (grid-cell difference plus FP32 offset difference, in
// grid-cell units, minimum image); its error is below Delta = 1e-5 (F_k + 1) for
// distances of a few grid cells, so every seed of the exact top k has an approximate
// key <= tau = F_k + 2 Delta (F_k: the k-th approximate key). The rings stop once the
// unvisited seeds are beyond tau + Delta. The entries <= tau then get the exact FP64 key
// (no FMA, ties by caller index) and are ranked exactly. If the K + 8 entries do not
// all fit below tau (many near ties, as on a lattice), the query takes the exact
// search instead. FAST = false (k > 24, where the unrolled lists would cost more
// registers than they save): the exact search for every query.
template <int K, bool FAST>
__global__ void __launch_bounds__(128) knn_kernel(const Pos4* __restrict__ pos,
                                                  const float4* __restrict__ off,
                                                  const int32_t* __restrict__ cellc,
                                                  const int32_t* __restrict__ cell_start,
                                                  KnnParams p, int32_t* __restrict__ knn,
                                                  double* __restrict__ d2k,
                                                  int* __restrict__ flags) {
    constexpr int K2 = K + 8;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= p.N) return;
    const int k = p.k;
    if (!FAST) {  // large k: the exact search only
        TopK<K> top;
        knn_exact<K>(pos, cell_start, p, q, top);
#pragma unroll
        for (int t = 0; t < K; t++) {
            if (t < k) knn[q * k + t] = top.s[t];
            if (t == k - 1) d2k[q] = top.d[t];
        }
        if (top.d[0] == 0.0) atomicOr(flags, 1);
        if (top.s[0] < 0) atomicOr(flags, 2);
        return;
    }
    const float4 oi = off[q];
    const int lc = cellc[q];
    const int c[3] = {lc & 1023, (lc >> 10) & 1023, (lc >> 20) & 1023};
    const float G[3] = {(float)p.G[0], (float)p.G[1], (float)p.G[2]};
    // grid cells are near-cubic; distances in units of the x cell size
    const float sy = (float)(p.h[1] / p.h[0]), sz = (float)(p.h[2] / p.h[0]);
    float fd[K2];
    int fi[K2];
#pragma unroll
    for (int t = 0; t < K2; t++) {
        fd[t] = FLT_MAX;
        fi[t] = -1;
    }
    const float m = fminf(fminf(fminf(oi.x, 1.f - oi.x), fminf(oi.y, 1.f - oi.y) * sy),
                          fminf(oi.z, 1.f - oi.z) * sz);
    const int Gmin = min(p.G[0], min(p.G[1], p.G[2]));
    bool ok = false;
    float tau = FLT_MAX;
    for (int r = 0;; r++) {
        if (2 * r + 1 > Gmin) break;  // rings would wrap: exact search
        for (int oz = -r; oz <= r; oz++) {
            const int cz = ((c[2] + oz) % p.G[2] + p.G[2]) % p.G[2];
            for (int oy = -r; oy <= r; oy++) {
                const int cy = ((c[1] + oy) % p.G[1] + p.G[1]) % p.G[1];
                const bool face = (oz == -r || oz == r || oy == -r || oy == r);
                const int step = (face || r == 0) ? 1 : 2 * r;
                for (int ox = -r; ox <= r; ox += step) {
                    const int cx = ((c[0] + ox) % p.G[0] + p.G[0]) % p.G[0];
                    const int64_t cell = ((int64_t)cz * p.G[1] + cy) * p.G[0] + cx;
                    const int32_t b = cell_start[cell], e = cell_start[cell + 1];
                    for (int32_t t = b; t < e; t++) {
                        if (t == q) continue;
                        const float4 oj = off[t];
                        float dx = (float)ox + (oj.x - oi.x);
                        float dy = (float)oy + (oj.y - oi.y);
                        float dz = (float)oz + (oj.z - oi.z);
                        if (dx > 0.5f * G[0]) dx -= G[0];
                        else if (dx < -0.5f * G[0]) dx += G[0];
                        if (dy > 0.5f * G[1]) dy -= G[1];
                        else if (dy < -0.5f * G[1]) dy += G[1];
                        if (dz > 0.5f * G[2]) dz -= G[2];
                        else if (dz < -0.5f * G[2]) dz += G[2];
                        dy *= sy;
                        dz *= sz;
                        const float d2 = dx * dx + dy * dy + dz * dz;
                        if (d2 < fd[K2 - 1]) {
#pragma unroll
                            for (int u = K2 - 1; u >= 0; u--) {
                                if (d2 < fd[u]) {
                                    const bool sh = u > 0 && d2 < fd[u - 1];
                                    fd[u] = sh ? fd[u - 1] : d2;
                                    fi[u] = sh ? fi[u - 1] : t;
                                }
                            }
                        }
                    }
                }
            }
        }
        float Fk = FLT_MAX;
#pragma unroll
        for (int t = 0; t < K2; t++)
            if (t == k - 1) Fk = fd[t];
        if (Fk == FLT_MAX) continue;
        const float delta = 1e-5f * (Fk + 1.f);
        tau = Fk + 2.f * delta;
        // every unvisited seed lies at least r + m cell sizes away
        const float bound = fminf((float)r * fminf(1.f, fminf(sy, sz)) + m, 1e30f);
        if (tau + delta < bound * bound * (1.f - 1e-6f)) {
            ok = true;
            break;
        }
    }
    TopK<K> top;
    if (ok && fd[K2 - 1] <= tau) ok = false;  // too many near ties for the list
    if (ok) {
        const Pos4 yi = pos[q];
        top.init();
#pragma unroll
        for (int u = 0; u < K2; u++)
            if (fd[u] <= tau && fi[u] >= 0) {
                const Pos4 yj = pos[fi[u]];
                top.insert(dist2_exact(yi, yj, p), (int)yj.w, fi[u]);
            }
    } else {
        knn_exact<K>(pos, cell_start, p, q, top);
    }
#pragma unroll
    for (int t = 0; t < K; t++) {
        if (t < k) knn[q * k + t] = top.s[t];
        if (t == k - 1) d2k[q] = top.d[t];
    }
    if (top.d[0] == 0.0) atomicOr(flags, 1);  // duplicate position
    if (top.s[0] < 0) atomicOr(flags, 2);      // fewer than k other seeds
}

int build_knn(DeviceState& d, cudaStream_t s, int* dup_flag_host) {
    NvtxRange nv("knn");
    KnnParams p;
    for (int a = 0; a < 3; a++) {
        p.G[a] = d.grid.G[a];
        p.h[a] = d.grid.h[a];
        p.L[a] = d.L[a];
        p.halfL[a] = 0.5 * d.L[a];
    }
    p.N = d.N;
    p.k = d.k;
    int* flags = (int*)(d.counters + 3);
    SDOT_CUDA_TRY(cudaMemsetAsync(flags, 0, 4, s));
    // FP32 grid-local offsets and grid cells: posf and leafc serve as scratch here (the
    // first Laguerre evaluation rewrites both)
    const unsigned nb = (unsigned)((d.N + 127) / 128);
    knn_prep_kernel<<<nb, 128, 0, s>>>(d.pos, d.N, p, d.posf, d.leafc);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
#define SDOT_KNN_LAUNCH(KK, F)                                                           \
    knn_kernel<KK, F><<<nb, 128, 0, s>>>(d.pos, d.posf, d.leafc, d.grid.cell_start, p, \
                                         d.knn, d.knn_d2k, flags)
    if (d.k <= 8) SDOT_KNN_LAUNCH(8, true);
    else if (d.k <= 16) SDOT_KNN_LAUNCH(16, true);
    else if (d.k <= 24) SDOT_KNN_LAUNCH(24, true);
    else if (d.k <= 32) SDOT_KNN_LAUNCH(32, false);
    else SDOT_KNN_LAUNCH(64, false);
#undef SDOT_KNN_LAUNCH
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    int h = 0;
    SDOT_CUDA_TRY(cudaMemcpyAsync(&h, flags, 4, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    *dup_flag_host = h;
    return SDOT_OK;
}

__global__ void knn_user_kernel(const int32_t* __restrict__ knn, const int32_t* __restrict__ perm,
                                int64_t N, int k, int32_t* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * k) return;
    int64_t s = t / k;
    int r = (int)(t - s * k);
    out[(int64_t)perm[s] * k + r] = perm[knn[t]];
}

int knn_to_user(const DeviceState& d, int32_t* out, cudaStream_t s) {
    int64_t n = d.N * d.k;
    knn_user_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d.knn, d.perm, d.N, d.k, out);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    return SDOT_OK;
}

}  // namespace sdot
