// After the solve: the Kantorovich potential at tau_I on a mesh and the mass density of
// the cells moved to an intermediate time (Sec. "Monge-Ampere-Kantorovich
// Reconstruction", the Legendre transform of psi and the last paragraph; Fig. 1).
//
//  - phi_I(q) = min_i [1/2 |q - x_i|^2 - psi_i], attained in the Laguerre cell i(q) that
//    contains q: every cell claims the mesh points inside it (planes tested with a small
//    tolerance, so a point on a facet is claimed by both cells), the smallest value of
//    its own 1/2 |q - x_i|^2 - psi_i wins (integer atomic minimum on the value's ordered
//    bits), then the claimants holding exactly that value take the owner by an integer
//    minimum on their (caller) index. The value is computed in the order
//    ((dx^2 + dy^2) + dz^2) / 2 - psi_i with correctly rounded operations.
//  - The Zel'dovich map q -> q + lambda (x_i - q) (lambda = D(tau)/D(tau_F)) shrinks cell
//    i about x_i by 1 - lambda and carries its mass nu_i uniformly. The mass of voxel v
//    is sum_i nu_i |V_i cap h_i^-1(v)| / |V_i| with h_i that homothety: each cell is
//    clipped by the six planes of every pulled-back voxel its moved bounding box meets.
//    The masses are summed in 64-bit fixed point (unit: 2^-62 of the box's mass, so no
//    voxel can overflow), so the sum does not depend on the order of the atomic
//    additions.
//
// One warp per cell. The cell is rebuilt in FP64 (seed frame, large polytope) from the
// facets of the context's last evaluation, which are its complete neighbour set.
#include <math.h>

#include <string>

#include "cell.cuh"

namespace sdot {

struct MeshParams {
    int M;                           // mesh points (voxels) per axis
    int pass;                        // 0: deposit and phi minimum, 1: owner
    double s;                        // 1 - lambda
    double h[3];                     // voxel size
    double mass_unit;                // fixed-point unit of the voxel masses
    const double* nu;                // masses (sorted order)
    unsigned long long* mass_fx;     // M^3 voxel masses (fixed point), or null
    unsigned long long* phi_ord;     // M^3 ordered bits of phi, or null
    int32_t* owner;                  // M^3 owner (caller index), or null (pass 1 only)
    int32_t* flags;                  // [0] cells that could not be rebuilt
    int32_t* work;                   // work counter
};

__device__ __forceinline__ unsigned long long d2ord(double f) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(f);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord2d(unsigned long long u) {
    return __longlong_as_double(
        (long long)((u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u));
}
__device__ __forceinline__ int wrap_index(long long v, int M) {
    long long r = v % M;
    return (int)(r < 0 ? r + M : r);
}
// minimum-image component, the rule of the oracle: if dx > L/2 subtract L, else if
// dx < -L/2 add L
__device__ __forceinline__ double wrap_rn(double dx, double L) {
    if (dx > __dmul_rn(0.5, L)) return __dsub_rn(dx, L);
    if (dx < -__dmul_rn(0.5, L)) return __dadd_rn(dx, L);
    return dx;
}

using MeshCap = CapL;
constexpr int MESH_WARPS = 2;

__global__ void __launch_bounds__(MESH_WARPS * 32)
    mesh_kernel(const __grid_constant__ ClipParams cp, const __grid_constant__ MeshParams mp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using PolyT = Poly<double, MeshCap>;
    PolyT* polys = reinterpret_cast<PolyT*>(smem_raw);
    const int lane = threadIdx.x & 31;
    PolyT& P = polys[2 * (threadIdx.x >> 5)];
    PolyT& Q = polys[2 * (threadIdx.x >> 5) + 1];
    const int M = mp.M;
    while (true) {
        int64_t i = 0;
        if (lane == 0) i = atomicAdd(mp.work, 1);
        i = __shfl_sync(FULLMASK, i, 0);
        if (i >= cp.N) break;
        CellCtx cc;
        cc.i = i;
        cc.yi = cp.pos[i];
        cc.psii = cp.psi[i];
        cc.si = load_seed(cp, i);
        cc.fr = seed_frame();
        bool bad = false;
        poly_init(P, cp, cc.fr.z, lane);
        const int nf = min(cp.fcnt[i], FCAP);
        const int rc = clip_list(P, cp, cc, cp.fcol + i * FCAP, nf, lane, bad);
        if (rc == CLIP_EMPTY || rc == CLIP_CAP || bad) {
            if (lane == 0) atomicAdd(mp.flags, 1);
            continue;
        }
        // bounding box of the cell (seed frame, units of a)
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int s = lane; s < P.nt; s += 32) {
            const double v[3] = {P.vx[s], P.vy[s], P.vz[s]};
            for (int a = 0; a < 3; a++) {
                lo[a] = fmin(lo[a], v[a]);
                hi[a] = fmax(hi[a], v[a]);
            }
        }
        for (int a = 0; a < 3; a++)
            for (int o = 16; o > 0; o >>= 1) {
                lo[a] = fmin(lo[a], __shfl_xor_sync(FULLMASK, lo[a], o));
                hi[a] = fmax(hi[a], __shfl_xor_sync(FULLMASK, hi[a], o));
            }
        const double y[3] = {cc.yi.x, cc.yi.y, cc.yi.z};
        const int32_t caller = (int32_t)cc.yi.w;
        // --- point location: the mesh points inside the cell --------------------------
        if (mp.phi_ord) {
            long long m0[3], m1[3];
            for (int a = 0; a < 3; a++) {
                m0[a] = (long long)ceil((y[a] + cp.a * lo[a]) / mp.h[a] - 0.5 - 1e-9);
                m1[a] = (long long)floor((y[a] + cp.a * hi[a]) / mp.h[a] - 0.5 + 1e-9);
            }
            const long long nx = m1[0] - m0[0] + 1, ny = m1[1] - m0[1] + 1,
                            nz = m1[2] - m0[2] + 1;
            const long long npts = (nx > 0 && ny > 0 && nz > 0) ? nx * ny * nz : 0;
            for (long long t = lane; t < npts; t += 32) {
                const long long mm[3] = {m0[0] + t % nx, m0[1] + (t / nx) % ny,
                                         m0[2] + t / (nx * ny)};
                int w[3];
                double q[3], p[3];
                for (int a = 0; a < 3; a++) {
                    w[a] = wrap_index(mm[a], M);
                    q[a] = __ddiv_rn(__dmul_rn((double)w[a] + 0.5, cp.L[a]), (double)M);
                    p[a] = wrap_rn(__dsub_rn(q[a], y[a]), cp.L[a]);
                }
                // inside every plane of the cell (units of a), with a tolerance of the
                // terms involved
                bool in = true;
                const double pa[3] = {p[0] * cp.inv_a, p[1] * cp.inv_a, p[2] * cp.inv_a};
                for (int k = 0; k < P.np && in; k++) {
                    const V4<double> pl = P.pl[k];
                    const double sd = pa[0] * pl.x + pa[1] * pl.y + pa[2] * pl.z - pl.w;
                    const double sc = fabs(pl.w) + P.plen[k] * (fabs(pa[0]) + fabs(pa[1]) +
                                                                fabs(pa[2]));
                    if (sd > 1e-12 * sc) in = false;
                }
                if (!in) continue;
                double s2 = 0.0;
                for (int a = 0; a < 3; a++) s2 = __dadd_rn(s2, __dmul_rn(p[a], p[a]));
                const double f = __dsub_rn(__dmul_rn(0.5, s2), cc.psii);
                const int64_t m = ((int64_t)w[2] * M + w[1]) * M + w[0];
                if (mp.pass == 0) atomicMin(&mp.phi_ord[m], d2ord(f));
                else if (mp.phi_ord[m] == d2ord(f)) atomicMin(&mp.owner[m], caller);
            }
        }
        if (mp.pass != 0 || !mp.mass_fx) continue;
        // --- deposit: the cell against every pulled-back voxel it meets --------------
        const double volP = poly_volume(P, lane);
        if (!(volP > 0.0)) {
            if (lane == 0) atomicAdd(mp.flags, 1);
            continue;
        }
        long long v0[3], v1[3];
        for (int a = 0; a < 3; a++) {
            v0[a] = (long long)floor((y[a] + mp.s * cp.a * lo[a]) / mp.h[a]);
            v1[a] = (long long)floor((y[a] + mp.s * cp.a * hi[a]) / mp.h[a]);
        }
        const double nui = mp.nu[i];
        for (long long vz = v0[2]; vz <= v1[2]; vz++)
            for (long long vy = v0[1]; vy <= v1[1]; vy++)
                for (long long vx = v0[0]; vx <= v1[0]; vx++) {
                    const long long vv[3] = {vx, vy, vz};
                    poly_copy(Q, P, lane);
                    bool empty = false, qbad = false;
                    for (int a = 0; a < 3 && !empty; a++) {
                        // voxel [v h, (v + 1) h] pulled back: p in [(v h - y)/s, ((v+1) h - y)/s]
                        const double blo = ((double)vv[a] * mp.h[a] - y[a]) / (mp.s * cp.a);
                        const double bhi = ((double)(vv[a] + 1) * mp.h[a] - y[a]) / (mp.s * cp.a);
                        V4<double> pn;
                        pn.x = a == 0 ? 1.0 : 0.0;
                        pn.y = a == 1 ? 1.0 : 0.0;
                        pn.z = a == 2 ? 1.0 : 0.0;
                        pn.w = bhi;
                        int r = poly_clip(Q, pn, 1.0, -2, lane, qbad);
                        if (r == CLIP_EMPTY) empty = true;
                        if (r == CLIP_CAP) {
                            qbad = true;
                            empty = true;
                        }
                        if (empty) break;
                        pn.x = -pn.x;
                        pn.y = -pn.y;
                        pn.z = -pn.z;
                        pn.w = -blo;
                        r = poly_clip(Q, pn, 1.0, -2, lane, qbad);
                        if (r == CLIP_EMPTY) empty = true;
                        if (r == CLIP_CAP) {
                            qbad = true;
                            empty = true;
                        }
                    }
                    if (qbad && lane == 0) atomicAdd(mp.flags, 1);
                    if (empty) continue;
                    const double vq = poly_volume(Q, lane);
                    if (!(vq > 0.0)) continue;
                    if (lane == 0) {
                        const double c = nui * (vq / volP);
                        const unsigned long long u = (unsigned long long)llrint(c / mp.mass_unit);
                        const int64_t m = ((int64_t)wrap_index(vz, M) * M + wrap_index(vy, M)) * M +
                                          wrap_index(vx, M);
                        atomicAdd(&mp.mass_fx[m], u);
                    }
                    __syncwarp();
                }
    }
}

__global__ void mesh_init_kernel(int64_t n, unsigned long long* mass_fx,
                                 unsigned long long* phi_ord, int32_t* owner) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (mass_fx) mass_fx[t] = 0ull;
    if (phi_ord) phi_ord[t] = 0xffffffffffffffffull;
    if (owner) owner[t] = INT32_MAX;
}

__global__ void mesh_out_kernel(int64_t n, const unsigned long long* __restrict__ mass_fx,
                                double unit_per_vox, const unsigned long long* __restrict__ phi_ord,
                                double* __restrict__ rho, double* __restrict__ phi,
                                int32_t* __restrict__ missing) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (rho) rho[t] = (double)mass_fx[t] * unit_per_vox;
    if (phi_ord) {
        const unsigned long long u = phi_ord[t];
        if (u == 0xffffffffffffffffull) atomicAdd(missing, 1);  // no cell claimed the point
        if (phi) phi[t] = ord2d(u);
    }
}

// ClipParams for rebuilding the cells of context d from its facets (FP64, seed frame)
ClipParams mesh_clip_params(DeviceState& d);

int mesh_eval(DeviceState& d, int M, double lambda, double* rho_dev, double* phi_dev,
              int32_t* owner_dev, void* scratch, cudaStream_t s) {
    NvtxRange nv("mesh");
    const int64_t n = (int64_t)M * M * M;
    unsigned long long* mass_fx = rho_dev ? (unsigned long long*)scratch : nullptr;
    unsigned long long* phi_ord =
        (phi_dev || owner_dev) ? (unsigned long long*)scratch + (rho_dev ? n : 0) : nullptr;
    int32_t* flags = d.counters + 26;  // [26] rebuild failures, [27] unclaimed points
    int32_t* work = d.counters + 28;
    SDOT_CUDA_TRY(cudaMemsetAsync(d.counters + 26, 0, 3 * sizeof(int32_t), s));
    const unsigned nb = (unsigned)((n + 255) / 256);
    mesh_init_kernel<<<nb, 256, 0, s>>>(n, mass_fx, phi_ord, owner_dev);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    MeshParams mp;
    mp.M = M;
    mp.s = 1.0 - lambda;
    for (int a = 0; a < 3; a++) mp.h[a] = d.L[a] / M;
    mp.mass_unit = d.L[0] * d.L[1] * d.L[2] / 4611686018427387904.0;  // |box| / 2^62
    mp.nu = d.nu;
    mp.mass_fx = mass_fx;
    mp.phi_ord = phi_ord;
    mp.owner = owner_dev;
    mp.flags = flags;
    mp.work = work;
    ClipParams cp = mesh_clip_params(d);
    const size_t smem = 2 * sizeof(Poly<double, MeshCap>) * MESH_WARPS;
    static const cudaError_t attr = cudaFuncSetAttribute(
        mesh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    SDOT_CUDA_TRY(attr);
    const int blocks = 4 * num_sms();
    for (int pass = 0; pass < (owner_dev ? 2 : 1); pass++) {
        mp.pass = pass;
        SDOT_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(int32_t), s));
        mesh_kernel<<<blocks, MESH_WARPS * 32, smem, s>>>(cp, mp);
        note_launch();
        SDOT_CUDA_TRY(cudaGetLastError());
    }
    const double vox = mp.h[0] * mp.h[1] * mp.h[2];
    mesh_out_kernel<<<nb, 256, 0, s>>>(n, mass_fx, mp.mass_unit / vox, phi_ord, rho_dev,
                                       phi_dev, d.counters + 27);
    note_launch();
    SDOT_CUDA_TRY(cudaGetLastError());
    int32_t h[2];
    SDOT_CUDA_TRY(cudaMemcpyAsync(h, d.counters + 26, 8, cudaMemcpyDeviceToHost, s));
    SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h[0] > 0) {
        set_error("sdot_mesh: " + std::to_string(h[0]) +
                  " cell(s) could not be rebuilt from their facets or clipped by a voxel");
        return SDOT_ERR_CAPACITY;
    }
    if (h[1] > 0) {
        set_error("sdot_mesh: " + std::to_string(h[1]) + " mesh point(s) claimed by no cell");
        return SDOT_ERR_CUDA;
    }
    return SDOT_OK;
}

}  // namespace sdot
