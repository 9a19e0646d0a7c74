// Power spectrum of a periodic mesh: the estimator behind the fractional BAO signal
// d(k) = P_wig(k) / P_nw(k) - 1 of Sec. "BAO reconstruction" (Fig. 2), applied to the
// densities sdot_mesh deposits for a wiggle / no-wiggle pair.
//
// delta = rho / mean(rho) - 1 on an M^3 mesh of a cubic box of side L; delta_k is the
// discrete Fourier transform divided by M^3, P(k) = L^3 |delta_k|^2 at k = 2 pi n / L,
// and mode n != 0 goes into bin b = floor(|n| + 1/2) for 1 <= b <= nbins. Per bin: the
// mean P over the modes, their mean |k| and their count, every mode of the full
// transform counted once (the real-to-complex half holds each pair +-n once, except on
// the planes n_c = 0 and n_c = M/2, where both members are stored).
//
// The transform is cuFFT's double-precision real-to-complex 3D FFT (a plain library
// transform, loaded with dlopen on first use so that nothing else in the library depends
// on it). The binning is this file's: mean(rho) by a fixed-order reduction; per bin the
// largest |F_k|^2 (integer maximum on the bits), then the sum of |F_k|^2 / max as 64-bit
// fixed point (unit 2^-38 of the bin's maximum) and of |n| (unit 2^-28), so the result
// does not depend on the order of the atomic additions.
#include <dlfcn.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include <cufft.h>

#include "internal.cuh"

namespace sdot {

namespace {

struct CufftApi {
    cufftResult (*plan3d)(cufftHandle*, int, int, int, cufftType) = nullptr;
    cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
    cufftResult (*exec_d2z)(cufftHandle, cufftDoubleReal*, cufftDoubleComplex*) = nullptr;
    cufftResult (*destroy)(cufftHandle) = nullptr;
    bool ok = false;
};

const CufftApi& cufft_api() {
    static const CufftApi api = [] {
        CufftApi a;
        // by soname (already loaded, or on the loader's path), then in the toolkit
        std::vector<std::string> names = {"libcufft.so.12", "libcufft.so.13", "libcufft.so.11",
                                          "libcufft.so"};
        const char* home = getenv("CUDA_HOME");
        for (const std::string dir : {std::string(home ? home : "/usr/local/cuda") + "/lib64/",
                                      std::string("/usr/local/cuda/lib64/")})
            for (const char* n : {"libcufft.so.12", "libcufft.so.13", "libcufft.so"})
                names.push_back(dir + n);
        void* h = nullptr;
        for (const std::string& n : names)
            if ((h = dlopen(n.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return a;
        a.plan3d = reinterpret_cast<decltype(a.plan3d)>(dlsym(h, "cufftPlan3d"));
        a.set_stream = reinterpret_cast<decltype(a.set_stream)>(dlsym(h, "cufftSetStream"));
        a.exec_d2z = reinterpret_cast<decltype(a.exec_d2z)>(dlsym(h, "cufftExecD2Z"));
        a.destroy = reinterpret_cast<decltype(a.destroy)>(dlsym(h, "cufftDestroy"));
        a.ok = a.plan3d && a.set_stream && a.exec_d2z && a.destroy;
        return a;
    }();
    return api;
}

constexpr int SPEC_THREADS = 256;
// fixed-point units: a bin holds at most ~2^24 weighted modes (M <= 1024), so sums stay
// below 2^62: |F_k|^2 / bin max (<= 1) in 2^-38, |n| (<= 887) in 2^-28
constexpr double FIX_P = 274877906944.0;  // 2^38
constexpr double FIX_K = 268435456.0;     // 2^28

__global__ void mesh_sum_partial(const double* __restrict__ rho, int64_t n,
                                 double* __restrict__ part) {
    __shared__ double sh[SPEC_THREADS / 32];
    double v = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        v += rho[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < SPEC_THREADS / 32; w++) s += sh[w];
        part[blockIdx.x] = s;
    }
}

__global__ void mesh_sum_final(const double* __restrict__ part, int nb,
                               double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; b++) s += part[b];
        *out = s;
    }
}

// half-space mode t (layout M x M x (M/2 + 1), last index fastest): its |n|, bin (0:
// none) and weight (modes stored for both members of a pair count once)
__device__ __forceinline__ int mode_of(int64_t t, int M, int Mh, int nbins, double& nn,
                                       int& w) {
    const int ic = (int)(t % Mh);
    const int64_t r = t / Mh;
    const int ib = (int)(r % M), ia = (int)(r / M);
    const int na = ia <= M / 2 ? ia : ia - M;
    const int nb = ib <= M / 2 ? ib : ib - M;
    const double d2 = (double)na * na + (double)nb * nb + (double)ic * ic;
    nn = sqrt(d2);
    w = (ic == 0 || ((M & 1) == 0 && ic == M / 2)) ? 1 : 2;
    if (d2 == 0.0) return 0;
    const int b = (int)floor(nn + 0.5);
    return b <= nbins ? b : 0;
}

__global__ void spec_max_kernel(const cufftDoubleComplex* __restrict__ F, int M, int Mh,
                                int64_t nmode, int nbins,
                                unsigned long long* __restrict__ maxbits) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nmode;
         t += (int64_t)gridDim.x * blockDim.x) {
        double nn;
        int w;
        const int b = mode_of(t, M, Mh, nbins, nn, w);
        if (!b) continue;
        const double p = F[t].x * F[t].x + F[t].y * F[t].y;
        // p >= 0: its bit pattern orders like its value
        atomicMax(&maxbits[b - 1], (unsigned long long)__double_as_longlong(p));
    }
}

__global__ void spec_sum_kernel(const cufftDoubleComplex* __restrict__ F, int M, int Mh,
                                int64_t nmode, int nbins,
                                const unsigned long long* __restrict__ maxbits,
                                unsigned long long* __restrict__ psum,
                                unsigned long long* __restrict__ ksum,
                                unsigned long long* __restrict__ cnt) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nmode;
         t += (int64_t)gridDim.x * blockDim.x) {
        double nn;
        int w;
        const int b = mode_of(t, M, Mh, nbins, nn, w);
        if (!b) continue;
        const double p = F[t].x * F[t].x + F[t].y * F[t].y;
        const double pm = __longlong_as_double((long long)maxbits[b - 1]);
        const double q = pm > 0.0 ? p / pm : 0.0;
        atomicAdd(&psum[b - 1], (unsigned long long)llrint(q * FIX_P) * (unsigned long long)w);
        atomicAdd(&ksum[b - 1], (unsigned long long)llrint(nn * FIX_K) * (unsigned long long)w);
        atomicAdd(&cnt[b - 1], (unsigned long long)w);
    }
}

}  // namespace

}  // namespace sdot

using namespace sdot;

extern "C" int sdot_power_spectrum(const double* rho, int M, double L, int nbins, double* P,
                                   double* kmean, int64_t* nmodes, void* stream) {
    set_error("");
    if (!rho || !P || M < 2 || M > 1024 || !(L > 0.0) || !isfinite(L) || nbins < 1 ||
        nbins > 2 * M) {
        set_error("sdot_power_spectrum: need rho, P, 2 <= M <= 1024, a finite L > 0 and "
                  "1 <= nbins <= 2 M");
        return SDOT_ERR_ARG;
    }
    const CufftApi& fft = cufft_api();
    if (!fft.ok) {
        set_error("sdot_power_spectrum: libcufft could not be loaded");
        return SDOT_ERR_CUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)M * M * M;
    const int Mh = M / 2 + 1;
    const int64_t nmode = (int64_t)M * M * Mh;
    NvtxRange nv("power_spectrum");
    // device scratch: a copy of rho (an out-of-place real-to-complex transform may use its
    // input as work space), the transform, the reduction partials and the bins
    const int nb_sum = 4 * num_sms();
    double* in = nullptr;
    cufftDoubleComplex* F = nullptr;
    double* part = nullptr;
    unsigned long long* bins = nullptr;  // maxbits, psum, ksum, cnt: nbins each
    cufftHandle plan = 0;
    bool have_plan = false;
    int rc = SDOT_OK;
    auto fail = [&](int code, const std::string& msg) {
        set_error("sdot_power_spectrum: " + msg);
        rc = code;
    };
    do {
        if (cudaMalloc(&in, (size_t)n * 8) != cudaSuccess ||
            cudaMalloc(&F, (size_t)nmode * sizeof(cufftDoubleComplex)) != cudaSuccess ||
            cudaMalloc(&part, (size_t)(nb_sum + 1) * 8) != cudaSuccess ||
            cudaMalloc(&bins, (size_t)4 * nbins * 8) != cudaSuccess) {
            cudaGetLastError();
            fail(SDOT_ERR_OOM, "device allocation failed");
            break;
        }
        if (cudaMemcpyAsync(in, rho, (size_t)n * 8, cudaMemcpyDefault, s) != cudaSuccess ||
            cudaMemsetAsync(bins, 0, (size_t)4 * nbins * 8, s) != cudaSuccess) {
            fail(SDOT_ERR_CUDA, "copy of rho failed");
            break;
        }
        mesh_sum_partial<<<nb_sum, SPEC_THREADS, 0, s>>>(in, n, part);
        note_launch();
        mesh_sum_final<<<1, 32, 0, s>>>(part, nb_sum, part + nb_sum);
        note_launch();
        if (fft.plan3d(&plan, M, M, M, CUFFT_D2Z) != CUFFT_SUCCESS) {
            fail(SDOT_ERR_CUDA, "cufftPlan3d failed");
            break;
        }
        have_plan = true;
        if (fft.set_stream(plan, s) != CUFFT_SUCCESS || fft.exec_d2z(plan, in, F) != CUFFT_SUCCESS) {
            fail(SDOT_ERR_CUDA, "cufftExecD2Z failed");
            break;
        }
        const unsigned grid = (unsigned)(8 * num_sms());
        spec_max_kernel<<<grid, SPEC_THREADS, 0, s>>>(F, M, Mh, nmode, nbins, bins);
        note_launch();
        spec_sum_kernel<<<grid, SPEC_THREADS, 0, s>>>(F, M, Mh, nmode, nbins, bins,
                                                       bins + nbins, bins + 2 * nbins,
                                                       bins + 3 * nbins);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) {
            fail(SDOT_ERR_CUDA, "kernel launch failed");
            break;
        }
        std::vector<unsigned long long> h((size_t)4 * nbins);
        double sum = 0.0;
        if (cudaMemcpyAsync(h.data(), bins, h.size() * 8, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(&sum, part + nb_sum, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            fail(SDOT_ERR_CUDA, "read-back failed");
            break;
        }
        const double mean = sum / (double)n;
        if (!(mean > 0.0) || !isfinite(mean)) {
            fail(SDOT_ERR_ARG, "the mean of rho must be positive and finite");
            break;
        }
        // P = L^3 |F_k|^2 / (M^3 mean)^2 with F the unnormalised transform of rho
        const double norm = L * L * L / ((double)n * (double)n * mean * mean);
        for (int b = 0; b < nbins; b++) {
            const double c = (double)h[3 * nbins + b];
            double pm;
            memcpy(&pm, &h[b], 8);
            P[b] = c > 0 ? norm * pm * ((double)h[nbins + b] / FIX_P) / c : 0.0;
            if (kmean) kmean[b] = c > 0 ? 2.0 * M_PI / L * ((double)h[2 * nbins + b] / FIX_K) / c : 0.0;
            if (nmodes) nmodes[b] = (int64_t)h[3 * nbins + b];
        }
    } while (false);
    if (have_plan) fft.destroy(plan);
    cudaFree(in);
    cudaFree(F);
    cudaFree(part);
    cudaFree(bins);
    return rc;
}
