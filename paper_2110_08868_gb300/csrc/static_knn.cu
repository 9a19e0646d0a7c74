// sdot_knn_static: the kNN build of sdot_create without any device allocation.
//
// Some callers cannot allocate device memory on their path: code that runs inside
// another framework's memory pool or under a fixed device-memory budget, and
// latency-sensitive code for which cudaMalloc/cudaFree are off limits because they can
// synchronise the whole device. This entry point serves them: it builds the grid hash
// and the k-nearest-neighbour lists for up to SDOT_STATIC_MAX_N seeds with all scratch
// in one fixed device array declared in this file, and it calls neither cudaMalloc,
// cudaFree nor any allocating library routine. The caller passes the positions and
// the output buffer (both device memory).
//
// The array is a file-scope __device__ array: every GPU that loads the library holds
// it until the process exits. Host code cannot use the array's name as a device
// address, so the first call on each device (with that device current) looks its
// address up with cudaGetSymbolAddress and caches it; make that first call before any
// stream capture. All calls share the array and it keeps the last call's contents:
// calls whose work overlaps on the GPU (different streams, or different host threads)
// race on it and must be serialised by the caller.
#include <string.h>

#include <mutex>

#include "internal.cuh"

namespace sdot {

// sizes: grid cells <= seeds for the default seeds_per_leaf of 2
constexpr int64_t ST_N = SDOT_STATIC_MAX_N;
constexpr int ST_K = SDOT_STATIC_MAX_K;
constexpr size_t ST_align(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t ST_POS = 0;
constexpr size_t ST_PERM = ST_POS + ST_align(ST_N * sizeof(Pos4));
constexpr size_t ST_IPERM = ST_PERM + ST_align(ST_N * 4);
constexpr size_t ST_KNN = ST_IPERM + ST_align(ST_N * 4);
constexpr size_t ST_D2K = ST_KNN + ST_align(ST_N * ST_K * 4);
constexpr size_t ST_START = ST_D2K + ST_align(ST_N * 8);
constexpr size_t ST_OFF = ST_START + ST_align((ST_N + 1) * 4);  // FP32 grid offsets
constexpr size_t ST_CELLC = ST_OFF + ST_align(ST_N * 16);            // grid cells
constexpr size_t ST_COUNTERS = ST_CELLC + ST_align(ST_N * 4);
constexpr size_t ST_TEMP = ST_COUNTERS + 256;
// build_grid temp: keys (N), counts and fills (ncell each), a flag, then scan temp
constexpr size_t ST_TEMP_BYTES = ST_align(ST_N * 4) + 2 * ST_align(ST_N * 4) + 256 + 64 * 1024;
constexpr size_t ST_TOTAL = ST_TEMP + ST_TEMP_BYTES;

static __device__ __align__(256) unsigned char g_static_scratch[ST_TOTAL];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_addr[MAX_DEVICES] = {nullptr};

// device address of the scratch array on the current device (looked up once)
int static_scratch(unsigned char** out) {
    int dev = 0;
    SDOT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("sdot_knn_static: device ordinal out of range");
        return SDOT_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) {
            set_error(std::string("sdot_knn_static: cudaGetSymbolAddress: ") +
                      cudaGetErrorString(e));
            return SDOT_ERR_CUDA;
        }
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    return SDOT_OK;
}
}  // namespace
}  // namespace sdot

using namespace sdot;

extern "C" int sdot_knn_static(const double* pos, int64_t N, const double box[3], int k,
                               int32_t* nbr, void* stream) {
    set_error("");
    if (!pos || !box || !nbr || N < 2 || k < 1 || k > N - 1) {
        set_error("sdot_knn_static: need pos, box, nbr, N >= 2 and 1 <= k < N");
        return SDOT_ERR_ARG;
    }
    if (N > SDOT_STATIC_MAX_N || k > SDOT_STATIC_MAX_K) {
        set_error("sdot_knn_static: N must be <= " + std::to_string((long long)SDOT_STATIC_MAX_N) +
                  " and k <= " + std::to_string(SDOT_STATIC_MAX_K) +
                  " (fixed scratch); use sdot_create/sdot_knn for larger problems");
        return SDOT_ERR_ARG;
    }
    for (int a = 0; a < 3; a++)
        if (!(box[a] > 0) || !isfinite(box[a])) {
            set_error("sdot_knn_static: box lengths must be finite and positive");
            return SDOT_ERR_ARG;
        }
    int cur_dev = 0;
    SDOT_CUDA_TRY(cudaGetDevice(&cur_dev));
    for (const void* p : {(const void*)pos, (const void*)nbr}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            set_error("sdot_knn_static: pos and nbr must be device (or managed) memory");
            return SDOT_ERR_ARG;
        }
        // the kernels run on the current device against that device's scratch array;
        // memory of another device would be reached through peer access, if at all
        if (at.type == cudaMemoryTypeDevice && at.device != cur_dev) {
            set_error("sdot_knn_static: pos and nbr must live on the current device (device " +
                      std::to_string(cur_dev) + "), one of them is on device " +
                      std::to_string(at.device));
            return SDOT_ERR_ARG;
        }
    }
    unsigned char* base = nullptr;
    int rc = static_scratch(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    DeviceState d;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.k = k;
    for (int a = 0; a < 3; a++) d.L[a] = box[a];
    d.a = cbrt(box[0] * box[1] * box[2] / (double)N);
    d.pos = (Pos4*)(base + ST_POS);
    d.perm = (int32_t*)(base + ST_PERM);
    d.iperm = (int32_t*)(base + ST_IPERM);
    d.knn = (int32_t*)(base + ST_KNN);
    d.knn_d2k = (double*)(base + ST_D2K);
    d.grid.cell_start = (int32_t*)(base + ST_START);
    d.posf = (float4*)(base + ST_OFF);
    d.leafc = (int32_t*)(base + ST_CELLC);
    d.counters = (int32_t*)(base + ST_COUNTERS);
    // the grid of sdot_create's default (2 seeds per cell) never has more cells than
    // seeds, which the scratch layout assumes
    double h = cbrt(2.0 * box[0] * box[1] * box[2] / (double)N);
    int64_t ncell = 1;
    for (int a = 0; a < 3; a++) {
        double g = floor(box[a] / h);
        if (g < 1) g = 1;
        ncell *= (int64_t)g;
    }
    if (ncell > N) {
        set_error("sdot_knn_static: box aspect gives more grid cells than seeds");
        return SDOT_ERR_ARG;
    }
    if ((rc = build_grid(d, pos, 2.0, base + ST_TEMP, s, "sdot_knn_static"))) return rc;
    int kflags = 0;
    if ((rc = build_knn(d, s, &kflags))) return rc;
    if (kflags & 1) {
        set_error("sdot_knn_static: two seeds share a position");
        return SDOT_ERR_DUPLICATE;
    }
    if (kflags & 2) {
        set_error("sdot_knn_static: fewer than k other seeds");
        return SDOT_ERR_TOO_FEW;
    }
    if ((rc = knn_to_user(d, nbr, s))) return rc;
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    return SDOT_OK;
}
