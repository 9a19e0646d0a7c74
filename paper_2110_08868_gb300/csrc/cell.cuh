// One Laguerre cell per warp: the polytope, its clipping, the security walk and the
// integrals. Included by clip.cu only.
//
// Cell i of eq. (laguerrecell) in seed-local coordinates p = q - y_i is
//     P_i = { p : p.d_ij <= b_ij for all j },  d_ij = minimum image of y_j - y_i,
//     b_ij = 1/2 |d_ij|^2 + psi_i - psi_j,
// the lifted power bisectors of the neighbours. Lengths are in units of the spacing
// a = (|box|/N)^(1/3) and psi in units of a^2, so every quantity is O(1).
//
// The polytope lives in shared memory as planes plus vertices; each vertex is the
// "dual triangle" of the three planes through it, oriented so that det(n_a, n_b, n_c)
// > 0. Clipping by a new plane: the lanes classify the vertices (one ballot), the
// removed vertices' dual edges whose reverse edge is not removed form the boundary
// cycle, and every boundary edge (a -> b) yields the new vertex (a, b, new plane).
// Integration walks each face's vertex cycle and sums fan tetrahedra from the centre
// of the vertices' bounding box (volume, first moment, area vector).
//
// Security test. Every vertex v of the polytope lies in the ball B(c, Rc), and
// 1/2|v|^2 <= Mv at every point of the polytope (Mv: the largest value at a vertex,
// 1/2|v|^2 being convex). A seed j at offset d cuts only if 1/2|v - d|^2 - psi_j <
// 1/2|v|^2 - psi_i at some point v of the polytope, and 1/2|v - d|^2 >=
// 1/2 (|c - d| - Rc)_+^2 on the ball, so j cannot cut when
//     1/2 (|c - d| - Rc)_+^2 >= Mv + psi_j - psi_i.
// For a node of the psi pyramid (a box of grid cells with psi_j <= psimax) at
// distance u from the ball centre this holds for every seed inside when
//     1/2 (u - Rc)_+^2 >= Mv + psimax - psi_i,
// so the walk discards the node. The grid cells that survive are tested seed by seed
// (ball and bounding-box support, then an exact vertex classification).
#pragma once

#include <cuda_fp16.h>
#include <float.h>
#include <math.h>

#include "internal.cuh"

namespace sdot {

#define FULLMASK 0xffffffffu

template <typename R>
struct V3 {
    R x, y, z;
};
template <typename R>
struct V4 {
    R x, y, z, w;
};

// Capacities of one polytope. The first passes use the small one (occupancy); a cell
// that overflows it is re-clipped in FP64 with the large one.
template <int MP_, int MT_, int STK_>
struct Cap {
    static constexpr int MP = MP_;        // plane slots (the 6 box planes included)
    static constexpr int MT = MT_;        // vertex slots
    static constexpr int SL = MT_ / 32;   // vertex slots per lane
    static constexpr int MREM = MT_ / 2;  // vertices removed by one clip
    static constexpr int MNEW = MT_ / 2;  // vertices created by one clip
    static constexpr int STK = STK_;      // traversal stack entries
};
using CapS = Cap<64, 128, 256>;
using CapL = Cap<96, 192, 512>;

template <typename R, class C>
struct Poly {
    V4<R> pl[C::MP];          // plane p.n <= w (frame coordinates)
    R plen[C::MP];            // |n|
    int32_t pj[C::MP];        // neighbour (sorted index) or -1 for a box face
    uint32_t tri[C::MT];      // plane slots a | b << 8 | c << 16
    R vx[C::MT], vy[C::MT], vz[C::MT];
    union {
        struct {                        // clipping and the security walk
            uint32_t rem[C::MREM];      // removed vertices of a clip (tri | slot << 24)
            uint32_t ftri[C::MNEW];     // new vertices of a clip
            R fx[C::MNEW], fy[C::MNEW], fz[C::MNEW];
            uint32_t stack[C::STK];     // traversal stack (see traverse)
        };
        struct {                        // integration
            uint32_t fend[C::MP];       // per face: end of its entries in fent
            uint32_t fent[3 * C::MT];   // (x | y << 8 | vertex slot << 16) by face
            uint8_t fmap[C::MP];        // plane slot -> index in the stored topology
            R fa[C::MP];                // per face: facet coefficient A / |n|, or -1
        };
    };
    float sup[27];            // support max_v v.u over the 26 stencil directions u
    int np, nt;
    int ncert;                // seeds recorded for the cell's certificate (-1: too many)
#ifdef SDOT_COUNTERS
    uint32_t wc[8];           // work counters of the current cell (diagnostic builds)
#endif
};

// Work counters, compiled in only with -DSDOT_COUNTERS (diagnostic builds). The
// count argument is evaluated by lane 0 only, so it must not contain a warp vote.
// 0 clip calls, 1 cuts, 2 node tests, 3 leaf visits, 4 seed tests, 5 candidates,
// 6 cells, 7 pyramid-walk rounds
#ifdef SDOT_COUNTERS
#define WCOUNT(P, k, n)                                    \
    do {                                                   \
        if ((threadIdx.x & 31) == 0) (P).wc[k] += (n);     \
    } while (0)
#else
#define WCOUNT(P, k, n) \
    do {                \
    } while (0)
#endif

struct ClipParams {
    int64_t N;
    int k;
    double a, inv_a, inv_a2;
    double L[3], halfL[3];
    float Lt[3], halfLt[3];  // box in units of a
    float ht[3];             // grid cell size in units of a
    int G[3];
    const Pos4* pos;
    const float4* posf;
    const double* psi;
    const int32_t* knn;
    const double* knn_d2k;
    const int32_t* cell_start;
    Pyramid pyr;
    // outputs
    double* vol;
    double* m1;
    float* anchor;
    uint8_t* status;
    int32_t* fcnt;
    int32_t* fcol;
    double* fval;
    int32_t* queue_out;
    int32_t* queue_cnt;
    int32_t* q64_out;
    int32_t* q64_cnt;
    int32_t* work_counter;
    const int32_t* worklist;  // null: cells 0..nwork-1
    int64_t nwork;
    unsigned long long* counters64;  // diagnostic work counters (8)
    const float* pslo;               // low part of psi/a^2
    const uint4* ioff;               // grid-cell offsets, 32-bit fixed point
    float hfix[3];                   // cell size / a / 2^32 (fixed-point unit)
    const int32_t* leafc;            // grid cell of each seed, x | y << 10 | z << 20
    int facets_valid;                // fcnt/fcol hold the previous diagram's facets
    uint32_t* topo;                  // N * TOPO stored vertices (three plane indices)
    uint8_t* topo_n;                 // N stored vertex counts (0: none)
    float nsz[MAXLEV][3];            // node size per pyramid level, units of a
    int pass;                        // 1 security test, 2 re-queue, 3 FP64 re-clip
    // carried security certificates (see process_cell)
    float* cert_f;                   // N * CERT_F: ball centre, radius, M and w reserves
    uint16_t* cert_s;                // N * CERT_S: inflated supports, FP16 rounded up
    int32_t* cert_j;                 // N * CERT_NEAR: seeds to re-test
    uint8_t* cert_n;                 // N: their count, 0xff: no certificate
    const uint32_t* cert_dpsi;       // ordered max and min of psi - psi_prev (a^2)
    int32_t* cert_carried;           // cells certified by a carried certificate
    int cert_use;                    // record and use certificates (first pass)
};

__device__ __forceinline__ double wrapd(double dx, double L, double halfL) {
    if (dx > halfL) return dx - L;
    if (dx < -halfL) return dx + L;
    return dx;
}
__device__ __forceinline__ float wrapf(float dx, float L, float halfL) {
    if (dx > halfL) return dx - L;
    if (dx < -halfL) return dx + L;
    return dx;
}

__device__ __forceinline__ uint32_t pack3(uint32_t a, uint32_t b, uint32_t c) {
    return a | (b << 8) | (c << 16);
}
__device__ __forceinline__ bool has_edge(uint32_t t, uint32_t x, uint32_t y) {
    // does triangle t contain the directed edge x -> y
    uint32_t a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
    return (a == x && b == y) || (b == x && c == y) || (c == x && a == y);
}
__device__ __forceinline__ uint32_t lanes_below(int lane) {
    return (lane == 0) ? 0u : ((1u << lane) - 1u);
}

template <typename R>
__device__ __forceinline__ R warp_max(R v) {
    for (int o = 16; o > 0; o >>= 1) {
        R u = __shfl_xor_sync(FULLMASK, v, o);
        v = v > u ? v : u;
    }
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
    return v;
}
template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
    return v;
}

template <typename R, class C>
__device__ __forceinline__ V3<R> vert(const Poly<R, C>& P, int s) {
    V3<R> v;
    v.x = P.vx[s];
    v.y = P.vy[s];
    v.z = P.vz[s];
    return v;
}
template <typename R, class C>
__device__ __forceinline__ void set_vert(Poly<R, C>& P, int s, const V3<R>& v) {
    P.vx[s] = v.x;
    P.vy[s] = v.y;
    P.vz[s] = v.z;
}

// The periodic box around the seed: the bisectors of the cell's own images at
// +-Lt e_a, written relative to the frame origin z (zero: the seed itself).
template <typename R, class C>
__device__ void poly_init(Poly<R, C>& P, const ClipParams& cp, const float* z, int lane) {
    if (lane < 6) {
        int ax = lane >> 1;
        R s = (lane & 1) ? R(-1) : R(1);
        R Lt = (R)cp.Lt[ax];
        V4<R> pl;
        pl.x = ax == 0 ? s * Lt : R(0);
        pl.y = ax == 1 ? s * Lt : R(0);
        pl.z = ax == 2 ? s * Lt : R(0);
        pl.w = R(0.5) * Lt * Lt - s * Lt * (R)z[ax];
        P.pl[lane] = pl;
        P.plen[lane] = Lt;
        P.pj[lane] = -1;
    }
    if (lane < 8) {
        int sx = (lane & 1) ? 1 : -1, sy = (lane & 2) ? 1 : -1, sz = (lane & 4) ? 1 : -1;
        uint32_t X = sx > 0 ? 0 : 1, Y = sy > 0 ? 2 : 3, Z = sz > 0 ? 4 : 5;
        P.tri[lane] = (sx * sy * sz > 0) ? pack3(X, Y, Z) : pack3(X, Z, Y);
        P.vx[lane] = R(0.5) * (R)cp.Lt[0] * (R)sx - (R)z[0];
        P.vy[lane] = R(0.5) * (R)cp.Lt[1] * (R)sy - (R)z[1];
        P.vz[lane] = R(0.5) * (R)cp.Lt[2] * (R)sz - (R)z[2];
    }
    if (lane == 0) {
        P.np = 6;
        P.nt = 8;
    }
    __syncwarp();
}

// The vertex of planes (a, b, c) of t; well: the triple is well conditioned,
// det(n_a, n_b, n_c) > dtol |n_a| |n_b| |n_c|.
template <typename R, class C>
__device__ __forceinline__ V3<R> vertex_of(const Poly<R, C>& P, uint32_t t, R dtol, bool& well) {
    const V4<R> A = P.pl[t & 0xff], B = P.pl[(t >> 8) & 0xff], Cc = P.pl[(t >> 16) & 0xff];
    // n_b x n_c, n_c x n_a, n_a x n_b
    R bcx = B.y * Cc.z - B.z * Cc.y, bcy = B.z * Cc.x - B.x * Cc.z, bcz = B.x * Cc.y - B.y * Cc.x;
    R cax = Cc.y * A.z - Cc.z * A.y, cay = Cc.z * A.x - Cc.x * A.z, caz = Cc.x * A.y - Cc.y * A.x;
    R abx = A.y * B.z - A.z * B.y, aby = A.z * B.x - A.x * B.z, abz = A.x * B.y - A.y * B.x;
    R det = A.x * bcx + A.y * bcy + A.z * bcz;
    R inv = R(1) / det;
    V3<R> v;
    v.x = (A.w * bcx + B.w * cax + Cc.w * abx) * inv;
    v.y = (A.w * bcy + B.w * cay + Cc.w * aby) * inv;
    v.z = (A.w * bcz + B.w * caz + Cc.w * abz) * inv;
    R la = P.plen[t & 0xff], lb = P.plen[(t >> 8) & 0xff], lc = P.plen[(t >> 16) & 0xff];
    well = det > dtol * (la * lb * lc);
    return v;
}

// drop planes no vertex references any more; returns the number of planes left
template <typename R, class C>
__device__ __noinline__ int poly_gc(Poly<R, C>& P, int lane) {
    constexpr int NW = (C::MP + 31) / 32;
    uint32_t used[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) used[w] = 0;
    for (int s = lane; s < P.nt; s += 32) {
        uint32_t t = P.tri[s];
#pragma unroll
        for (int e = 0; e < 3; e++) {
            uint32_t q = (t >> (8 * e)) & 0xff;
#pragma unroll
            for (int w = 0; w < NW; w++)
                if ((q >> 5) == (uint32_t)w) used[w] |= 1u << (q & 31);
        }
    }
#pragma unroll
    for (int w = 0; w < NW; w++) used[w] = __reduce_or_sync(FULLMASK, used[w]);
    used[0] |= 0x3fu;  // box planes keep their slots
    int before[NW];
    int acc = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        before[w] = acc;
        acc += __popc(used[w]);
    }
    const int nn = acc;
    const int np = P.np;
    const uint32_t below = lanes_below(lane);
    // move the surviving planes down (read all, then write)
    V4<R> pl[NW];
    R len[NW];
    int32_t pj[NW];
    int dst[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) {
        int q = lane + 32 * w;
        dst[w] = -1;
        if (q < np && (used[w] >> lane & 1u)) {
            pl[w] = P.pl[q];
            len[w] = P.plen[q];
            pj[w] = P.pj[q];
            dst[w] = before[w] + __popc(used[w] & below);
        }
    }
    __syncwarp();
#pragma unroll
    for (int w = 0; w < NW; w++)
        if (dst[w] >= 0) {
            P.pl[dst[w]] = pl[w];
            P.plen[dst[w]] = len[w];
            P.pj[dst[w]] = pj[w];
        }
    __syncwarp();
    for (int s = lane; s < P.nt; s += 32) {
        uint32_t t = P.tri[s], r = 0;
#pragma unroll
        for (int e = 0; e < 3; e++) {
            uint32_t q = (t >> (8 * e)) & 0xff;
            uint32_t w = q >> 5, b = q & 31;
            uint32_t m = (b == 0) ? 0u : ((1u << b) - 1u);
            uint32_t nq = 0;
#pragma unroll
            for (int u = 0; u < NW; u++)
                if ((uint32_t)u == w) nq = before[u] + __popc(used[u] & m);
            r |= nq << (8 * e);
        }
        P.tri[s] = r;
    }
    __syncwarp();
    if (lane == 0) P.np = nn;
    __syncwarp();
    return nn;
}

enum { CLIP_NONE = 0, CLIP_CUT = 1, CLIP_EMPTY = 2, CLIP_CAP = 3 };

// relative tolerance of the vertex classification: a vertex counts as outside only
// when it is beyond the plane by more than this fraction of the terms involved, so
// planes that merely touch an edge or a corner (lattice-like degeneracy) do not cut
template <typename R>
__device__ __forceinline__ R class_eps() {
    return sizeof(R) == 4 ? R(2e-7) : R(1e-13);
}
template <typename R>
__device__ __forceinline__ bool beyond(const V3<R>& v, const V4<R>& pn, R plen, R& sd) {
    sd = v.x * pn.x + v.y * pn.y + v.z * pn.z - pn.w;
    R scale = fabs(pn.w) + plen * (fabs(v.x) + fabs(v.y) + fabs(v.z));
    return sd > class_eps<R>() * scale;
}

// Does the plane cut the polytope (some vertex strictly beyond it)? Warp-uniform.
template <typename R, class C>
__device__ __noinline__ bool poly_cut_by(const Poly<R, C>& P, const V4<R>& pn, R plen,
                                         int lane) {
    bool o = false;
    for (int q = lane; q < P.nt; q += 32) {
        R sd;
        o |= beyond(vert(P, q), pn, plen, sd);
    }
    return __any_sync(FULLMASK, o);
}

// Clip by p.n <= w (tag j). Non-finite geometry sets bad. Warp-uniform.
template <typename R, class C>
__device__ __noinline__ int poly_clip(Poly<R, C>& P, const V4<R>& pn, R plen, int32_t j,
                                      int lane, bool& bad) {
    constexpr int SL = C::SL;
    const int nt = P.nt;
    uint32_t m[SL];
    int nrem = 0;
#pragma unroll
    for (int t = 0; t < SL; t++) {
        const int s = lane + 32 * t;
        bool out = false;
        m[t] = 0u;
        if (32 * t < nt) {  // warp-uniform
            if (s < nt) {
                R sd;
                out = beyond(vert(P, s), pn, plen, sd);
            }
            m[t] = __ballot_sync(FULLMASK, out);
            nrem += __popc(m[t]);
        }
    }
    WCOUNT(P, 0, 1);
    if (nrem == 0) return CLIP_NONE;
    WCOUNT(P, 1, 1);
    if (nrem == nt) return CLIP_EMPTY;
    if (nrem > C::MREM) return CLIP_CAP;
    if (P.np >= C::MP) {
        if (poly_gc(P, lane) >= C::MP) return CLIP_CAP;
    }
    const uint32_t ps = (uint32_t)P.np;
    const uint32_t below = lanes_below(lane);
    // removed list: triangle | slot << 24
    {
        int base = 0;
#pragma unroll
        for (int t = 0; t < SL; t++) {
            if ((m[t] >> lane) & 1u)
                P.rem[base + __popc(m[t] & below)] =
                    P.tri[lane + 32 * t] | ((uint32_t)(lane + 32 * t) << 24);
            base += __popc(m[t]);
        }
    }
    if (lane == 0) {
        P.pl[ps] = pn;
        P.plen[ps] = plen;
        P.pj[ps] = j;
    }
    __syncwarp();
    // boundary edges of the removed region: dual edges whose reverse is not removed
    uint32_t bmask = 0;  // 3 bits per removed entry handled by this lane
    int cnt = 0;
    for (int r = lane, e = 0; r < nrem; r += 32, e++) {
        uint32_t t = P.rem[r] & 0xffffffu;
        uint32_t a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
        bool fab = false, fbc = false, fca = false;
        for (int q = 0; q < nrem; q++) {
            uint32_t u = P.rem[q] & 0xffffffu;
            fab |= has_edge(u, b, a);
            fbc |= has_edge(u, c, b);
            fca |= has_edge(u, a, c);
        }
        uint32_t bits = (fab ? 0u : 1u) | (fbc ? 0u : 2u) | (fca ? 0u : 4u);
        bmask |= bits << (3 * e);
        cnt += __popc(bits);
    }
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += y;
    }
    const int nnew = __shfl_sync(FULLMASK, incl, 31);
    const int nkept = nt - nrem;
    if (nkept + nnew > C::MT || nnew > C::MNEW) return CLIP_CAP;
    // new vertices: the point of the edge's two planes and the new plane; when that
    // system is ill-conditioned (the new plane almost parallel to the edge) the vertex
    // is interpolated on the edge between its kept and removed end points
    bool lbad = false;
    {
        int pos = incl - cnt;
        const R dtol = sizeof(R) == 4 ? R(1e-3) : R(1e-6);
        for (int r = lane, e = 0; r < nrem; r += 32, e++) {
            const uint32_t rr = P.rem[r];
            const uint32_t t = rr & 0xffffffu, sr = rr >> 24;
            const uint32_t bits = (bmask >> (3 * e)) & 7u;
            for (int k = 0; k < 3; k++) {
                if (!(bits >> k & 1u)) continue;
                const uint32_t x = (t >> (8 * k)) & 0xff, y = (t >> (8 * ((k + 1) % 3))) & 0xff;
                const uint32_t nt3 = pack3(x, y, ps);
                bool well;
                V3<R> v = vertex_of(P, nt3, dtol, well);
                if (!well) {
                    int sk = -1;
                    for (int q = 0; q < nt; q++) {
                        const bool o = (m[q >> 5] >> (q & 31)) & 1u;
                        if (!o && has_edge(P.tri[q], y, x)) {
                            sk = q;
                            break;
                        }
                    }
                    if (sk >= 0) {
                        V3<R> vk = vert(P, sk), vr = vert(P, sr);
                        R s_k, s_r;
                        beyond(vk, pn, plen, s_k);
                        beyond(vr, pn, plen, s_r);
                        R tt = R(0);
                        if (s_k < R(0) && s_r > s_k) tt = s_k / (s_k - s_r);
                        tt = tt < R(0) ? R(0) : (tt > R(1) ? R(1) : tt);
                        v.x = vk.x + tt * (vr.x - vk.x);
                        v.y = vk.y + tt * (vr.y - vk.y);
                        v.z = vk.z + tt * (vr.z - vk.z);
                    } else {
                        lbad = true;
                    }
                }
                if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) lbad = true;
                P.ftri[pos] = nt3;
                P.fx[pos] = v.x;
                P.fy[pos] = v.y;
                P.fz[pos] = v.z;
                pos++;
            }
        }
    }
    __syncwarp();
    // compact the kept vertices in place (read all, then write)
    {
        uint32_t kt[SL];
        V3<R> kv[SL];
        int dst[SL];
        int base = 0;
#pragma unroll
        for (int t = 0; t < SL; t++) {
            const int s = lane + 32 * t;
            dst[t] = -1;
            if (32 * t < nt) {  // warp-uniform
                const bool keep = s < nt && !((m[t] >> lane) & 1u);
                const uint32_t km = __ballot_sync(FULLMASK, keep);
                if (keep) {
                    kt[t] = P.tri[s];
                    kv[t] = vert(P, s);
                    dst[t] = base + __popc(km & below);
                }
                base += __popc(km);
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < SL; t++)
            if (dst[t] >= 0) {
                P.tri[dst[t]] = kt[t];
                set_vert(P, dst[t], kv[t]);
            }
    }
    __syncwarp();
    for (int n = lane; n < nnew; n += 32) {
        P.tri[nkept + n] = P.ftri[n];
        P.vx[nkept + n] = P.fx[n];
        P.vy[nkept + n] = P.fy[n];
        P.vz[nkept + n] = P.fz[n];
    }
    if (lane == 0) {
        P.np = ps + 1;
        P.nt = nkept + nnew;
    }
    if (__any_sync(FULLMASK, lbad)) bad = true;
    __syncwarp();
    return CLIP_CUT;
}

// is seed j already one of the polytope's planes? (warp-uniform j)
template <typename R, class C>
__device__ __forceinline__ bool has_plane(const Poly<R, C>& P, int32_t j, int lane) {
    bool dup = false;
    for (int q = lane; q < P.np; q += 32) dup |= P.pj[q] == j;
    return __any_sync(FULLMASK, dup);
}

// The cell's own seed in grid-local form: integer grid cell and FP32 offset from the
// grid cell's corner (units of a), psi/a^2 split into two floats (hi + lo).
struct SeedRef {
    int c[3];
    float off[3];
    uint32_t io[3];
    float phi, plo;
};

__device__ __forceinline__ SeedRef load_seed(const ClipParams& cp, int64_t i) {
    SeedRef r;
    float4 p = cp.posf[i];
    int lc = cp.leafc[i];
    r.c[0] = lc & 1023;
    r.c[1] = (lc >> 10) & 1023;
    r.c[2] = (lc >> 20) & 1023;
    r.off[0] = p.x;
    r.off[1] = p.y;
    r.off[2] = p.z;
    r.phi = p.w;
    r.plo = cp.pslo[i];
    uint4 q = cp.ioff[i];
    r.io[0] = q.x;
    r.io[1] = q.y;
    r.io[2] = q.z;
    return r;
}

// Frame of the FP32 polytope of one cell: origin z (units of a, relative to the
// seed), snapped to multiples of 2^-12 grid cells so that z is exact in FP64 and
// nearly so in FP32.
struct Frame {
    float z[3];    // z in FP32
    double zd[3];  // z in FP64
};

__device__ __forceinline__ Frame make_frame(const ClipParams& cp, const float* zwant) {
    Frame f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float za = zwant[a];
        if (!isfinite(za)) za = 0.f;
        za = fminf(fmaxf(za, -cp.halfLt[a]), cp.halfLt[a]);
        // snapped to a multiple of q = ht / 4096 (the nearest one up to FP32 rounding of
        // the quotient; any multiple serves, the choice is deterministic)
        const double q = (double)cp.ht[a] * (1.0 / 4096.0);
        f.zd[a] = (double)llrintf(za * (4096.f / cp.ht[a])) * q;
        f.z[a] = (float)f.zd[a];
    }
    return f;
}

// the frame at the seed itself (FP64 cells)
__device__ __forceinline__ Frame seed_frame() {
    Frame f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        f.z[a] = 0.f;
        f.zd[a] = 0.0;
    }
    return f;
}

// plane of neighbour j for cell i, built in FP64 (normalised units, seed frame)
__device__ __forceinline__ void make_plane(const ClipParams& cp, const Pos4& yi, double psii,
                                           int32_t j, double& nx, double& ny, double& nz,
                                           double& w) {
    Pos4 yj = cp.pos[j];
    nx = wrapd(yj.x - yi.x, cp.L[0], cp.halfL[0]) * cp.inv_a;
    ny = wrapd(yj.y - yi.y, cp.L[1], cp.halfL[1]) * cp.inv_a;
    nz = wrapd(yj.z - yi.z, cp.L[2], cp.halfL[2]) * cp.inv_a;
    w = 0.5 * (nx * nx + ny * ny + nz * nz) + (psii - cp.psi[j]) * cp.inv_a2;
}

// FP32 plane of seed j for cell i in the cell's frame, q.d <= 1/2 |d|^2 - d.z + psi_i -
// psi_j with p = z + q. The seed difference is taken exactly: grid-cell difference
// and 32-bit fixed-point offsets combine into one int64 per axis (minimum image on
// the fixed-point period G 2^32). The normal d is rounded once to FP32, which moves
// the plane by at most one rounding of |d| |q| at a vertex q of the cell; the offset
// is summed in FP64 from the exact d and the hi + lo psi, then rounded once, so it
// carries one rounding of its own (small) size: neither the distance of the cell
// from its seed nor the size of d - z enters the error.
__device__ __forceinline__ void plane_fix(const ClipParams& cp, const SeedRef& si,
                                          const Frame& fr, int32_t j, float& nx, float& ny,
                                          float& nz, float& w) {
    int lc = cp.leafc[j];
    uint4 q = cp.ioff[j];
    int cj[3] = {lc & 1023, (lc >> 10) & 1023, (lc >> 20) & 1023};
    uint32_t oj[3] = {q.x, q.y, q.z};
    float d[3];
    double t = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int dc = cj[a] - si.c[a];
        if (2 * dc > cp.G[a]) dc -= cp.G[a];
        else if (2 * dc < -cp.G[a]) dc += cp.G[a];
        long long di = ((long long)dc << 32) + (long long)oj[a] - (long long)si.io[a];
        const long long per = (long long)cp.G[a] << 32;
        if (2 * di > per) di -= per;
        else if (2 * di < -per) di += per;
        d[a] = (float)di * cp.hfix[a];
        const double dd = (double)di * (double)cp.hfix[a];
        t = fma(dd, fma(0.5, dd, -fr.zd[a]), t);
    }
    nx = d[0];
    ny = d[1];
    nz = d[2];
    float4 pj = cp.posf[j];
    const double dphi =
        ((double)si.phi - (double)pj.w) + ((double)si.plo - (double)cp.pslo[j]);
    w = (float)(t + dphi);
}

// FP32 plane of seed j for cell i from grid-local coordinates (seed frame): the
// integer part of the difference is exact, so the plane is accurate to FP32 relative
// precision of |d| and of the psi difference (psi carried as hi + lo floats). Used
// only by the conservative prefilters, which allow for that rounding.
__device__ __forceinline__ void plane_f32(const ClipParams& cp, const SeedRef& si, int32_t j,
                                          float& nx, float& ny, float& nz, float& w) {
    float4 pj = cp.posf[j];
    int lc = cp.leafc[j];
    int cj[3] = {lc & 1023, (lc >> 10) & 1023, (lc >> 20) & 1023};
    float oj[3] = {pj.x, pj.y, pj.z};
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int dc = cj[a] - si.c[a];
        if (2 * dc > cp.G[a]) dc -= cp.G[a];
        else if (2 * dc < -cp.G[a]) dc += cp.G[a];
        float v = (float)dc * cp.ht[a] + (oj[a] - si.off[a]);
        d[a] = wrapf(v, cp.Lt[a], cp.halfLt[a]);
    }
    nx = d[0];
    ny = d[1];
    nz = d[2];
    w = 0.5f * (nx * nx + ny * ny + nz * nz) + ((si.phi - pj.w) + (si.plo - cp.pslo[j]));
}

// Current bounds of the polytope (seed-relative coordinates, units of a): box
// [bmin, bmax], its centre c, the radius Rc of the ball around c holding every
// vertex, and Mv = max over the vertices of 1/2 |v|^2.
struct Bounds {
    float zf[3];  // frame origin of the polytope's vertices (relative to the seed)
    float bmin[3], bmax[3];
    float c[3];
    float Rc;
    float Mv;
    float cabs[3];  // c in absolute coordinates, wrapped into the box
    float yabs[3];  // the seed in absolute coordinates
    float psi_i;    // psi_i / a^2 (hi part)
};

// order-preserving map of a float onto uint32, so a warp max runs on integers
__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// x wrapped into [0, Lt) as fmodf then one period added to a negative remainder would
// give it. The polytope's centre lies within half a box of its seed, so x is in
// (-Lt, 2 Lt), where one subtraction (exact, Sterbenz) or addition does it; any other
// x takes the general path, kept out of line.
static __device__ __noinline__ float wrap_box_slow(float x, float Lt) {
    x = fmodf(x, Lt);
    if (x < 0.f) x += Lt;
    return x >= Lt ? 0.f : x;
}
__device__ __forceinline__ float wrap_box(float x, float Lt) {
    if (x >= Lt && x < 2.f * Lt) x -= Lt;
    else if (x < 0.f && x > -Lt) x += Lt;
    else if (!(x >= 0.f && x < Lt)) return wrap_box_slow(x, Lt);
    return x >= Lt ? 0.f : x;
}

// Bounds of the polytope (seed-relative coordinates): its support in the 26 directions
// u with components in {-1, 0, 1}, sup[(ux + 1) + 3 (uy + 1) + 9 (uz + 1)] = max_v v.u,
// the bounding box (the supports in the axis directions, exact), the largest |v|^2 (Mv),
// and the ball around the box centre c holding every vertex (Rc). Lane k < 27 owns
// direction k (lane 13, the zero direction, takes |v|^2) and scans every vertex from
// shared memory: one loop, no reductions for the 26 directions.
template <typename R, class C>
__device__ __noinline__ void poly_bounds(const Poly<R, C>& P, const ClipParams& cp, Bounds& b,
                                         int lane) {
    Poly<R, C>& Pm = const_cast<Poly<R, C>&>(P);
    const float ux = (float)(lane % 3 - 1), uy = (float)((lane / 3) % 3 - 1),
                uz = (float)(lane / 9 - 1);
    const float w2 = lane == 13 ? 1.f : 0.f;
    const float z0 = b.zf[0], z1 = b.zf[1], z2 = b.zf[2];
    const int nt = P.nt;
    float h = lane == 13 ? 0.f : -1e30f;
#pragma unroll 1
    for (int s = 0; s < nt; s++) {
        const float x = (float)P.vx[s] + z0, y = (float)P.vy[s] + z1, z = (float)P.vz[s] + z2;
        const float d = fmaf(ux, x, fmaf(uy, y, uz * z));
        h = fmaxf(h, fmaf(w2, fmaf(x, x, fmaf(y, y, z * z)), d));
    }
    if (lane < 27) Pm.sup[lane] = h;
    __syncwarp();
    // +x 14, -x 12, +y 16, -y 10, +z 22, -z 4
    const int ip[3] = {14, 16, 22}, in[3] = {12, 10, 4};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        b.bmax[a] = P.sup[ip[a]];
        b.bmin[a] = -P.sup[in[a]];
        b.c[a] = 0.5f * (b.bmin[a] + b.bmax[a]);
    }
    b.Mv = 0.5f * P.sup[13] * 1.0001f + 1e-6f;
    __syncwarp();
    if (lane == 0) Pm.sup[13] = 0.f;  // the zero direction (never used by the prefilter)
    float r2 = 0.f;
#pragma unroll 1
    for (int s = lane; s < nt; s += 32) {
        const float dx = ((float)P.vx[s] + z0) - b.c[0];
        const float dy = ((float)P.vy[s] + z1) - b.c[1];
        const float dz = ((float)P.vz[s] + z2) - b.c[2];
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
    }
    r2 = warp_max(r2);
    b.Rc = sqrtf(r2) * 1.0001f + 1e-5f;
#pragma unroll
    for (int a = 0; a < 3; a++) b.cabs[a] = wrap_box(b.yabs[a] + b.c[a], cp.Lt[a]);
    __syncwarp();
}

// distance from p to the interval [lo, lo + w] on a circle of length Lt
__device__ __forceinline__ float circ_gap(float p, float lo, float w, float Lt) {
    float t = p - lo;
    if (t < 0.f) t += Lt;
    if (t >= Lt) t -= Lt;
    if (t <= w) return 0.f;
    return fminf(t - w, Lt - t);
}

// True when no seed of node (X, Y, Z) of a pyramid level can cut the polytope:
// 1/2 (u - Rc)_+^2 >= Mv + psimax - psi_i with u the distance from the ball centre
// to the node's box (see the head of this file). The level (its psimax row pmax, node
// counts d and node size sz) and the ball (centre c in absolute coordinates, Rc, Mv,
// psi_i) come in registers: the walk loads them once, not per node.
struct WalkBall {
    float c[3];
    float Rc, Mv, psi_i;
};

__device__ __forceinline__ WalkBall walk_ball(const Bounds& b) {
    WalkBall w;
    w.c[0] = b.cabs[0];
    w.c[1] = b.cabs[1];
    w.c[2] = b.cabs[2];
    w.Rc = b.Rc;
    w.Mv = b.Mv;
    w.psi_i = b.psi_i;
    return w;
}

__device__ __forceinline__ bool node_pruned(const float* __restrict__ pmax, const int d[3],
                                            const float sz[3], const float Lt[3],
                                            const WalkBall& wb, int X, int Y, int Z) {
    const float pm = pmax[(int64_t)((Z * d[1] + Y) * d[0] + X)];
    if (pm == -INFINITY) return true;  // no seed inside
    const int c[3] = {X, Y, Z};
    float u2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        // the last node of an axis ends at the box edge
        const float lo = (float)c[a] * sz[a];
        const float w = (c[a] + 1 == d[a]) ? Lt[a] - lo : sz[a];
        const float g = circ_gap(wb.c[a], lo, w, Lt[a]);
        u2 += g * g;
    }
    const float du = fmaxf(sqrtf(u2) * (1.f - 1e-6f) - wb.Rc, 0.f);
    const float lhs = 0.5f * du * du;
    const float rhs = wb.Mv + (pm - wb.psi_i);
    const float margin = 2e-5f * (lhs + wb.Mv + fabsf(pm) + fabsf(wb.psi_i)) + 1e-5f;
    return lhs - rhs > margin;
}

// Conservative FP32 test: can the plane (n, w) of a seed (seed frame) reach the
// polytope? Two valid upper bounds of max_vertex v.n are used and the plane is a
// candidate only if both reach it. (1) With |n| sorted, n1 >= n2 >= n3 on axes a1, a2,
// a3, n = n3 u3 + (n2 - n3) u2 + (n1 - n2) u1 for the stencil directions u1 = s1 e_a1,
// u2 = u1 + s2 e_a2, u3 = u2 + s3 e_a3 (s: the signs of n), nonnegative coefficients,
// so by sublinearity of the support h, h(n) <= n3 h(u3) + (n2 - n3) h(u2) +
// (n1 - n2) h(u1); this is never weaker than the bounding box's support. (2) The ball
// of radius Rc around the box centre c: h(n) <= c.n + Rc |n|.
__device__ __forceinline__ bool support_may_cut(const float* sup, const Bounds& b, float nx,
                                                float ny, float nz, float w) {
    float m[3] = {fabsf(nx), fabsf(ny), fabsf(nz)};
    int code[3] = {nx >= 0.f ? 1 : -1, ny >= 0.f ? 3 : -3, nz >= 0.f ? 9 : -9};
    // sort descending (three compare-exchanges)
#define SDOT_CX(i, j)                                  \
    if (m[i] < m[j]) {                                 \
        const float tm = m[i];                         \
        m[i] = m[j];                                   \
        m[j] = tm;                                     \
        const int tc = code[i];                        \
        code[i] = code[j];                             \
        code[j] = tc;                                  \
    }
    SDOT_CX(0, 1)
    SDOT_CX(1, 2)
    SDOT_CX(0, 1)
#undef SDOT_CX
    const int k1 = 13 + code[0], k2 = k1 + code[1], k3 = k2 + code[2];
    const float t3 = m[2] * sup[k3], t2 = (m[1] - m[2]) * sup[k2], t1 = (m[0] - m[1]) * sup[k1];
    const float S = t1 + t2 + t3;
    const float margin = 2e-5f * (fabsf(t1) + fabsf(t2) + fabsf(t3) + fabsf(w)) + 1e-5f;
    if (!(S > w - margin)) return false;
    const float cn = b.c[0] * nx + b.c[1] * ny + b.c[2] * nz;
    const float rn = b.Rc * sqrtf(nx * nx + ny * ny + nz * nz);
    const float margin2 = 2e-5f * (fabsf(cn) + rn + fabsf(w)) + 1e-5f;
    return cn + rn > w - margin2;
}

// Carried security certificates. A pass-1 walk that certifies a cell records, besides
// the cell itself, a certificate for later evaluations: the walk's node tests use the
// ball inflated by CERT_EPS and M inflated by CERT_ETA, and every seed that is not a
// plane of the cell and passes the prefilter inflated the same way (supports + CERT_EPS
// rounded up to FP16, ball radius + CERT_EPS, offset w - CERT_ETA) is recorded for an
// exact re-test. At a later evaluation the certificate holds, and the walk is skipped,
// when the warm-started polytope lies inside the stored ball and below the stored
// supports, its M fits the stored M less the change of psi differences since, the
// stored w reserve covers that change, and no recorded seed cuts it exactly: every seed
// a node test excluded still satisfies 1/2 (u - R)_+^2 >= M + psi_j - psi_i, and every
// seed the inflated prefilter excluded still has its plane beyond the stored supports.
constexpr float CERT_EPS = 0.01f;  // ball radius and support reserve, units of a
constexpr float CERT_ETA = 0.01f;  // reserve for the change of psi_j - psi_i, units of a^2

// inflated support of direction k as stored (FP16, rounded up)
__device__ __forceinline__ float cert_sup(const float* sup, int k) {
    return __half2float(__float2half_ru(__fadd_ru(sup[k], CERT_EPS)));
}

// The prefilter of support_may_cut on the inflated certificate quantities.
__device__ __forceinline__ bool cert_may_cut(const float* sup, const Bounds& b, float nx,
                                             float ny, float nz, float w) {
    float m[3] = {fabsf(nx), fabsf(ny), fabsf(nz)};
    int code[3] = {nx >= 0.f ? 1 : -1, ny >= 0.f ? 3 : -3, nz >= 0.f ? 9 : -9};
#define SDOT_CX(i, j)                                  \
    if (m[i] < m[j]) {                                 \
        const float tm = m[i];                         \
        m[i] = m[j];                                   \
        m[j] = tm;                                     \
        const int tc = code[i];                        \
        code[i] = code[j];                             \
        code[j] = tc;                                  \
    }
    SDOT_CX(0, 1)
    SDOT_CX(1, 2)
    SDOT_CX(0, 1)
#undef SDOT_CX
    const int k1 = 13 + code[0], k2 = k1 + code[1], k3 = k2 + code[2];
    const float t3 = m[2] * cert_sup(sup, k3), t2 = (m[1] - m[2]) * cert_sup(sup, k2),
                t1 = (m[0] - m[1]) * cert_sup(sup, k1);
    const float wr = __fsub_rd(w, CERT_ETA);
    const float S = t1 + t2 + t3;
    const float margin = 2e-5f * (fabsf(t1) + fabsf(t2) + fabsf(t3) + fabsf(wr)) + 1e-5f;
    if (!(S > wr - margin)) return false;
    const float R = __fadd_ru(b.Rc, CERT_EPS);
    const float cn = b.c[0] * nx + b.c[1] * ny + b.c[2] * nz;
    const float rn = R * sqrtf(nx * nx + ny * ny + nz * nz);
    const float margin2 = 2e-5f * (fabsf(cn) + rn + fabsf(wr)) + 1e-5f;
    return cn + rn > wr - margin2;
}

enum { MODE_CERTIFY = 0, MODE_FULL = 1 };
enum { LEAF_OK = 0, LEAF_STOP = 1 };

struct CellCtx {
    int64_t i;
    Pos4 yi;      // FP64 seed (FP64 planes)
    double psii;  // FP64 psi_i
    SeedRef si;   // grid-local seed (FP32 planes)
    Frame fr;     // frame of the polytope (the seed itself for FP64 cells)
};

// exact plane of seed j in the polytope's frame (per lane)
template <typename R>
__device__ __forceinline__ void build_plane(const ClipParams& cp, const CellCtx& cc, int32_t j,
                                            V4<R>& pn, R& plen) {
    if (sizeof(R) == 8) {
        double nxd, nyd, nzd, wd;
        make_plane(cp, cc.yi, cc.psii, j, nxd, nyd, nzd, wd);
        pn.x = (R)nxd;
        pn.y = (R)nyd;
        pn.z = (R)nzd;
        pn.w = (R)wd;
    } else {
        float nx, ny, nz, w;
        plane_fix(cp, cc.si, cc.fr, j, nx, ny, nz, w);
        pn.x = (R)nx;
        pn.y = (R)ny;
        pn.z = (R)nz;
        pn.w = (R)w;
    }
    plen = sqrt(pn.x * pn.x + pn.y * pn.y + pn.z * pn.z);
}

template <typename R>
__device__ __forceinline__ V4<R> shfl_plane(const V4<R>& p, int src) {
    V4<R> q;
    q.x = __shfl_sync(FULLMASK, p.x, src);
    q.y = __shfl_sync(FULLMASK, p.y, src);
    q.z = __shfl_sync(FULLMASK, p.z, src);
    q.w = __shfl_sync(FULLMASK, p.w, src);
    return q;
}

// The seeds of up to 32 grid cells (leaf < 0: none), spread evenly over the lanes:
// each seed passes the conservative prefilter in its lane, the survivors are checked
// exactly one by one (warp-uniform). CERTIFY stops at the first seed that cuts; FULL
// clips it. Returns LEAF_STOP when the cell's processing must stop.
template <typename R, class C, int MODE>
__device__ __noinline__ int process_leaves(Poly<R, C>& P, const ClipParams& cp,
                                           const CellCtx& cc, Bounds& b, int64_t leaf, int lane,
                                           bool& bad, uint32_t& st) {
    int32_t sb = 0;
    int n = 0;
    if (leaf >= 0) {
        sb = cp.cell_start[leaf];
        n = cp.cell_start[leaf + 1] - sb;
    }
#ifdef SDOT_COUNTERS
    {
        const uint32_t nleaf = __popc(__ballot_sync(FULLMASK, leaf >= 0));
        WCOUNT(P, 3, nleaf);
    }
#endif
    int incl = n;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(FULLMASK, incl, 31);
    const int excl = incl - n;
    WCOUNT(P, 4, total);
    // a certifying walk of the first pass records the cell's certificate
    const bool rec = MODE == MODE_CERTIFY && cp.pass == 1 && cp.cert_use;
    for (int base = 0; base < total; base += 32) {
        const int t = base + lane;
        // the lane q owning flattened seed t: the first with incl[q] > t
        int q = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int y = __shfl_sync(FULLMASK, incl, q + step - 1);
            if (y <= t) q += step;
        }
        const int ex = __shfl_sync(FULLMASK, excl, q);
        const int32_t s0 = __shfl_sync(FULLMASK, sb, q);
        const int32_t s = s0 + (t - ex);
        bool cand = false, nearb = false;
        if (t < total && s != (int32_t)cc.i) {
            float nx, ny, nz, w;
            plane_f32(cp, cc.si, s, nx, ny, nz, w);
            cand = support_may_cut(P.sup, b, nx, ny, nz, w);
            if (rec) nearb = cand || cert_may_cut(P.sup, b, nx, ny, nz, w);
        }
        uint32_t cm = __ballot_sync(FULLMASK, cand);
        uint32_t nm = rec ? __ballot_sync(FULLMASK, nearb) : cm;
        WCOUNT(P, 5, __popc(cm));
        if (!nm) continue;
        // drop the seeds that already are planes of the polytope (the cell's own facet
        // neighbours pass the prefilter), then build the exact planes of the rest
        for (uint32_t m2 = nm; m2;) {
            const int src = __ffs(m2) - 1;
            m2 &= m2 - 1;
            if (has_plane(P, __shfl_sync(FULLMASK, s, src), lane)) {
                cm &= ~(1u << src);
                nm &= ~(1u << src);
            }
        }
        // the certificate's seeds to re-test (P.ftri is free during a certifying walk)
        if (rec && nm) {
            const int n0 = P.ncert;
            const int k = __popc(nm);
            __syncwarp();
            if (n0 >= 0 && n0 + k <= CERT_NEAR) {
                if ((nm >> lane) & 1u) P.ftri[n0 + __popc(nm & lanes_below(lane))] = (uint32_t)s;
                if (lane == 0) P.ncert = n0 + k;
            } else if (lane == 0) {
                P.ncert = -1;
            }
            __syncwarp();
        }
        if (!cm) continue;
        cand = (cm >> lane) & 1u;
        V4<R> pl;
        pl.x = pl.y = pl.z = pl.w = R(0);
        R len = R(1);
        if (cand) build_plane(cp, cc, s, pl, len);
        while (cm) {
            const int src = __ffs(cm) - 1;
            cm &= cm - 1;
            const int32_t j = __shfl_sync(FULLMASK, s, src);
            const V4<R> pn = shfl_plane(pl, src);
            const R plen = __shfl_sync(FULLMASK, len, src);
            // an earlier clip of this round may have added the same seed? (seeds are
            // distinct within a round, so only FULL mode's clips can change the set)
            if (MODE == MODE_FULL && has_plane(P, j, lane)) continue;
            if (MODE == MODE_CERTIFY) {
                if (poly_cut_by(P, pn, plen, lane)) {
                    st |= CS_UNCERTIFIED;
                    return LEAF_STOP;
                }
                continue;
            }
            const int rc = poly_clip(P, pn, plen, j, lane, bad);
            if (rc == CLIP_EMPTY) {
                st |= CS_EMPTY;
                return LEAF_STOP;
            }
            if (rc == CLIP_CAP) {
                st |= CS_CAPACITY | CS_CAP_POLY;
                return LEAF_STOP;
            }
            if (rc == CLIP_CUT) poly_bounds(P, cp, b, lane);
        }
    }
    return LEAF_OK;
}

// Near-first pass for re-queued cells: the grid cells in Chebyshev rings around the
// grid cell of the previous centroid, so the polytope is small before the pyramid
// walk (which visits nodes in no particular order) starts.
template <typename R, class C>
__device__ __noinline__ bool ring_walk(Poly<R, C>& P, const ClipParams& cp, const CellCtx& cc,
                                       Bounds& b, const float* zprev, int lane, bool& bad,
                                       uint32_t& st) {
    int ca[3];
    float hmin = 1e30f;
    for (int a = 0; a < 3; a++) {
        float za = fmodf(b.yabs[a] + zprev[a], cp.Lt[a]);
        if (za < 0.f) za += cp.Lt[a];
        int c = (int)floorf(za / cp.ht[a]);
        ca[a] = c < 0 ? 0 : (c >= cp.G[a] ? cp.G[a] - 1 : c);
        hmin = fminf(hmin, cp.ht[a]);
    }
    const int Gmin = min(cp.G[0], min(cp.G[1], cp.G[2]));
    for (int r = 0; r <= 3; r++) {
        if (2 * r + 1 > Gmin) break;
        if (r >= 2 && (float)(r - 1) * hmin > 2.f * b.Rc) break;
        const int w = 2 * r + 1, n3 = w * w * w;
        for (int base = 0; base < n3; base += 32) {
            const int t = base + lane;
            int64_t leaf = -1;
            if (t < n3) {
                const int ox = t % w - r, oy = (t / w) % w - r, oz = t / (w * w) - r;
                const int ch = max(abs(ox), max(abs(oy), abs(oz)));
                if (ch == r) {
                    const int cx = ((ca[0] + ox) % cp.G[0] + cp.G[0]) % cp.G[0];
                    const int cy = ((ca[1] + oy) % cp.G[1] + cp.G[1]) % cp.G[1];
                    const int cz = ((ca[2] + oz) % cp.G[2] + cp.G[2]) % cp.G[2];
                    leaf = ((int64_t)cz * cp.G[1] + cy) * cp.G[0] + cx;
                }
            }
            if (process_leaves<R, C, MODE_FULL>(P, cp, cc, b, leaf, lane, bad, st) == LEAF_STOP)
                return false;
        }
    }
    return true;
}

// Walk the pyramid. MODE_CERTIFY: return false as soon as a seed cuts the polytope.
// MODE_FULL: clip every such seed. Returns true when the walk completed. A stack entry
// is a node to expand: level << 27 | Z << 18 | Y << 9 | X (levels >= 1 have at most
// 256 nodes per axis); its children are the up to 4 x 4 x 4 nodes one level down. The
// root is the virtual node (nlev, 0, 0, 0) whose children are the top level.
__device__ __forceinline__ uint32_t pack_node(int l, int x, int y, int z) {
    return ((uint32_t)l << 27) | ((uint32_t)z << 18) | ((uint32_t)y << 9) | (uint32_t)x;
}

template <typename R, class C, int MODE>
__device__ __noinline__ bool traverse(Poly<R, C>& P, const ClipParams& cp, const CellCtx& cc,
                                      Bounds& b, int lane, bool& bad, uint32_t& st) {
    if (lane == 0) P.stack[0] = pack_node(cp.pyr.nlev, 0, 0, 0);
    int sp = 1;
    const float Lt[3] = {cp.Lt[0], cp.Lt[1], cp.Lt[2]};
    WalkBall wb = walk_ball(b);
    if (MODE == MODE_CERTIFY && cp.pass == 1 && cp.cert_use) {
        // the certificate's reserves (the same roundings as cert_store)
        wb.Rc = __fadd_ru(wb.Rc, CERT_EPS);
        wb.Mv = __fadd_ru(wb.Mv, CERT_ETA);
    }
    __syncwarp();
    while (sp > 0) {
        const uint32_t e = P.stack[sp - 1];
        sp--;
        __syncwarp();
        const int cl = (int)(e >> 27) - 1;  // level of the children
        const int x0 = 4 * (int)(e & 511u), y0 = 4 * (int)((e >> 9) & 511u),
                  z0 = 4 * (int)((e >> 18) & 511u);
        const int cd[3] = {cp.pyr.dim[cl][0], cp.pyr.dim[cl][1], cp.pyr.dim[cl][2]};
        const float csz[3] = {cp.nsz[cl][0], cp.nsz[cl][1], cp.nsz[cl][2]};
        const float* pmax = cp.pyr.psimax + cp.pyr.off[cl];
        // rounds of 32 children; a round is skipped when none of its children exists
        const int nzr = min(4, cd[2] - z0);  // child layers along z (2 per round)
        WCOUNT(P, 7, 1);
        for (int base = 0; base < 16 * nzr; base += 32) {
            const int t = base + lane;
            const int cx = x0 + (t & 3), cy = y0 + ((t >> 2) & 3), cz = z0 + (t >> 4);
            bool surv = false;
            if (cx < cd[0] && cy < cd[1] && cz < cd[2])
                surv = !node_pruned(pmax, cd, csz, Lt, wb, cx, cy, cz);
            WCOUNT(P, 2, 32);
            const uint32_t sm = __ballot_sync(FULLMASK, surv);
            if (sm == 0) continue;
            if (cl > 0) {
                const int n = __popc(sm);
                if (sp + n > C::STK) {
                    st |= CS_CAPACITY | CS_CAP_STACK;
                    return false;
                }
                if (surv) P.stack[sp + __popc(sm & lanes_below(lane))] = pack_node(cl, cx, cy, cz);
                sp += n;
                __syncwarp();
                continue;
            }
            // surviving grid cells: their seeds
            const int64_t leaf = surv ? ((int64_t)cz * cp.G[1] + cy) * cp.G[0] + cx : -1;
            if (process_leaves<R, C, MODE>(P, cp, cc, b, leaf, lane, bad, st) == LEAF_STOP)
                return false;
            if (MODE == MODE_FULL) wb = walk_ball(b);  // a clip may have shrunk the polytope
        }
    }
    return true;
}

// Integrate the polytope and write the outputs of cell i; cen receives the centroid
// relative to the seed (units of a, every lane) and the return value says whether it
// is valid (positive finite volume).
template <typename R, class C>
__device__ __noinline__ bool integrate(Poly<R, C>& P, const ClipParams& cp, const Frame& fr,
                                       int64_t i, int lane, bool& bad, uint32_t& st,
                                       float* cen) {
    // volume and first moment: summed per face in R, the face totals in FP64; the
    // surface closure check and the facet areas in R
    double vol6 = 0, mx = 0, my = 0, mz = 0;
    R sx = 0, sy = 0, sz = 0, sabs = 0;
    // FP32 consistency check (degenerate facets): two facet planes that meet at a vertex
    // while their normals are less than ANGLE_MIN apart (the bisectors of seeds packed in
    // a clump, seen from a cell a few spacings away) meet in an edge whose FP32 position
    // is off by about (plane rounding) / angle, far above the cell's own rounding; such a
    // cell fails the check and is clipped again in FP64. Box planes take no part.
    if (sizeof(R) == 4) {
        constexpr float SIN2_MIN = 0.03f * 0.03f;  // ANGLE_MIN = 0.03 rad
        bool ill = false;
#pragma unroll 1
        for (int s2 = lane; s2 < P.nt; s2 += 32) {
            const uint32_t t = P.tri[s2];
            const uint32_t ia = t & 0xff, ib = (t >> 8) & 0xff, ic = (t >> 16) & 0xff;
            const V4<R> A = P.pl[ia], Bq = P.pl[ib], Cq = P.pl[ic];
            const float la2 = A.x * A.x + A.y * A.y + A.z * A.z;
            const float lb2 = Bq.x * Bq.x + Bq.y * Bq.y + Bq.z * Bq.z;
            const float lc2 = Cq.x * Cq.x + Cq.y * Cq.y + Cq.z * Cq.z;
            const float bcx = Bq.y * Cq.z - Bq.z * Cq.y, bcy = Bq.z * Cq.x - Bq.x * Cq.z,
                        bcz = Bq.x * Cq.y - Bq.y * Cq.x;
            const float cax = Cq.y * A.z - Cq.z * A.y, cay = Cq.z * A.x - Cq.x * A.z,
                        caz = Cq.x * A.y - Cq.y * A.x;
            const float abx = A.y * Bq.z - A.z * Bq.y, aby = A.z * Bq.x - A.x * Bq.z,
                        abz = A.x * Bq.y - A.y * Bq.x;
            if (ia >= 6 && ib >= 6 && abx * abx + aby * aby + abz * abz < SIN2_MIN * la2 * lb2)
                ill = true;
            if (ib >= 6 && ic >= 6 && bcx * bcx + bcy * bcy + bcz * bcz < SIN2_MIN * lb2 * lc2)
                ill = true;
            if (ic >= 6 && ia >= 6 && cax * cax + cay * cay + caz * caz < SIN2_MIN * lc2 * la2)
                ill = true;
        }
        if (__any_sync(FULLMASK, ill)) bad = true;
    }
    // apex of the tetrahedron fans: the centre o of the vertices' bounding box, so the
    // determinants involve offsets of the cell's own size even when the cell lies far
    // from its seed (no cancellation of large terms in FP32)
    R o[3];
    {
        R mn[3] = {R(1e30), R(1e30), R(1e30)}, mxv[3] = {R(-1e30), R(-1e30), R(-1e30)};
#pragma unroll 1
        for (int s2 = lane; s2 < P.nt; s2 += 32) {
            const R v[3] = {P.vx[s2], P.vy[s2], P.vz[s2]};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                mn[a] = fmin(mn[a], v[a]);
                mxv[a] = fmax(mxv[a], v[a]);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
            for (int q = 16; q > 0; q >>= 1) {
                mn[a] = fmin(mn[a], __shfl_xor_sync(FULLMASK, mn[a], q));
                mxv[a] = fmax(mxv[a], __shfl_xor_sync(FULLMASK, mxv[a], q));
            }
            o[a] = R(0.5) * (mn[a] + mxv[a]);
        }
    }
    const int nt = P.nt;
    const int np = P.np;
    // bucket the vertices by face: vertex s = (a, b, c) lies on faces a, b and c, and
    // on face a the cycle continues from it along (b, c). Counts, an exclusive scan
    // over the faces, then the entries (their order inside a face is immaterial: the
    // walk below starts at the entry of the lowest vertex slot). After the fill,
    // fend[f] is the end of face f's entries and the start of face f + 1's.
#pragma unroll 1
    for (int f = lane; f < np; f += 32) P.fend[f] = 0u;
    __syncwarp();
#pragma unroll 1
    for (int s2 = lane; s2 < nt; s2 += 32) {
        const uint32_t t = P.tri[s2];
        atomicAdd(&P.fend[t & 0xff], 1u);
        atomicAdd(&P.fend[(t >> 8) & 0xff], 1u);
        atomicAdd(&P.fend[(t >> 16) & 0xff], 1u);
    }
    __syncwarp();
    {
        uint32_t carry = 0;
#pragma unroll 1
        for (int f0 = 0; f0 < np; f0 += 32) {
            const int f = f0 + lane;
            const uint32_t c = f < np ? P.fend[f] : 0u;
            uint32_t incl = c;
            for (int q = 1; q < 32; q <<= 1) {
                const uint32_t y = __shfl_up_sync(FULLMASK, incl, q);
                if (lane >= q) incl += y;
            }
            if (f < np) P.fend[f] = carry + incl - c;  // start, advanced by the fill
            carry += __shfl_sync(FULLMASK, incl, 31);
        }
    }
    __syncwarp();
#pragma unroll 1
    for (int s2 = lane; s2 < nt; s2 += 32) {
        const uint32_t t = P.tri[s2];
        const uint32_t a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
        const uint32_t sv = (uint32_t)s2 << 16;
        P.fent[atomicAdd(&P.fend[a], 1u)] = b | (c << 8) | sv;
        P.fent[atomicAdd(&P.fend[b], 1u)] = c | (a << 8) | sv;
        P.fent[atomicAdd(&P.fend[c], 1u)] = a | (b << 8) | sv;
    }
    __syncwarp();
    int nf = 0;  // facets among this lane's faces
#pragma unroll 1
    for (int f = lane; f < np; f += 32) {
        const int e0 = f > 0 ? (int)P.fend[f - 1] : 0;
        const int m = (int)P.fend[f] - e0;
        P.fa[f] = R(-1);
        if (m == 0) continue;
        if (m < 3) {
            bad = true;
            continue;
        }
        // fan apex: the entry of the lowest vertex slot
        int first = e0;
        for (int e = e0 + 1; e < e0 + m; e++)
            if ((P.fent[e] >> 16) < (P.fent[first] >> 16)) first = e;
        // walk the cycle: the entry after (x, y) is the one whose x equals y
        uint32_t ecur = P.fent[first];
        const uint32_t x0 = ecur & 0xff;
        V3<R> v0 = vert(P, ecur >> 16);
        v0.x -= o[0];
        v0.y -= o[1];
        v0.z -= o[2];
        V3<R> vp = v0;
        R Sx = 0, Sy = 0, Sz = 0;
        R fv6 = 0, fmx = 0, fmy = 0, fmz = 0;
        bool ok = true;
        for (int step = 1; step < m; step++) {
            const uint32_t yv = (ecur >> 8) & 0xff;
            int nxt = -1;
            for (int e = e0; e < e0 + m; e++)
                if ((P.fent[e] & 0xff) == yv) {
                    nxt = e;
                    break;
                }
            if (nxt < 0 || nxt == first) {
                ok = false;
                break;
            }
            ecur = P.fent[nxt];
            V3<R> vc = vert(P, ecur >> 16);
            vc.x -= o[0];
            vc.y -= o[1];
            vc.z -= o[2];
            if (step >= 2) {
                // fan triangle (v0, vp, vc) and tetrahedron (o, v0, vp, vc)
                const R ax = vp.x - v0.x, ay = vp.y - v0.y, az = vp.z - v0.z;
                const R bx = vc.x - v0.x, by = vc.y - v0.y, bz = vc.z - v0.z;
                const R cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
                Sx += cx;
                Sy += cy;
                Sz += cz;
                // 6 |tet(o, v0, vp, vc)| = det(v0, vp, vc) with vertices relative to o
                const R d6 = v0.x * cx + v0.y * cy + v0.z * cz;
                fv6 += d6;
                fmx += d6 * (v0.x + vp.x + vc.x);
                fmy += d6 * (v0.y + vp.y + vc.y);
                fmz += d6 * (v0.z + vp.z + vc.z);
            }
            vp = vc;
        }
        if (ok && ((ecur >> 8) & 0xff) != x0) ok = false;
        if (!ok) {
            bad = true;
            continue;
        }
        vol6 += (double)fv6;
        mx += (double)fmx;
        my += (double)fmy;
        mz += (double)fmz;
        const R ax2 = R(0.5) * Sx, ay2 = R(0.5) * Sy, az2 = R(0.5) * Sz;
        const R A = sqrt(ax2 * ax2 + ay2 * ay2 + az2 * az2);
        sx += ax2;
        sy += ay2;
        sz += az2;
        sabs += A;
        if (P.pj[f] >= 0 && A > R(0)) {
            P.fa[f] = A / P.plen[f];
            nf++;
        }
    }
    vol6 = warp_sum(vol6);
    mx = warp_sum(mx);
    my = warp_sum(my);
    mz = warp_sum(mz);
    sx = warp_sum_r(sx);
    sy = warp_sum_r(sy);
    sz = warp_sum_r(sz);
    sabs = warp_sum_r(sabs);
    // facets, in the order lane by lane, then this lane's faces in slot order
    int incl = nf;
    for (int q = 1; q < 32; q <<= 1) {
        const int y = __shfl_up_sync(FULLMASK, incl, q);
        if (lane >= q) incl += y;
    }
    const int total = __shfl_sync(FULLMASK, incl, 31);
    // plane slot -> index in [the 6 box planes, then the facets as written], for the
    // stored topology (0xff: the slot has no facet)
    uint8_t* map = P.fmap;
#pragma unroll 1
    for (int f = lane; f < np; f += 32) map[f] = f < 6 ? (uint8_t)f : (uint8_t)0xff;
    __syncwarp();
    if (total > FCAP) {
        st |= CS_CAPACITY | CS_CAP_FACE;
    } else {
        int pos = incl - nf;
#pragma unroll 1
        for (int f = lane; f < np; f += 32) {
            const R c = P.fa[f];
            if (!(c >= R(0))) continue;
            cp.fcol[i * FCAP + pos] = P.pj[f];
            cp.fval[i * FCAP + pos] = (double)c * cp.a;
            map[f] = (uint8_t)(6 + pos);
            pos++;
        }
    }
    __syncwarp();
    // the topology: every vertex as three indices into that list (kept only when
    // every plane a vertex uses is a box plane or a facet, and the counts fit)
    bool tok = total <= FCAP && 6 + total <= CapS::MP && nt <= TOPO;
#pragma unroll 1
    for (int s2 = lane; s2 < nt && tok; s2 += 32) {
        const uint32_t t = P.tri[s2];
        const uint32_t a = map[t & 0xff], b2 = map[(t >> 8) & 0xff], c = map[(t >> 16) & 0xff];
        if ((a | b2 | c) == 0xffu || a == 0xff || b2 == 0xff || c == 0xff) tok = false;
        else cp.topo[i * TOPO + s2] = pack3(a, b2, c);
    }
    tok = __all_sync(FULLMASK, tok);
    const R closure = sqrt(sx * sx + sy * sy + sz * sz);
    const R tol = sizeof(R) == 4 ? R(1e-4) : R(1e-10);
    if (!(closure <= tol * sabs)) bad = true;
    const double vol = vol6 * (1.0 / 6.0);
    if (!(vol > 0.0) || !isfinite(vol)) bad = true;
    // first moment about the seed = moment about o + (z + o) V (mx.. hold 24 x moment
    // about o; o is relative to the frame origin z)
    mx += 24.0 * (fr.zd[0] + (double)o[0]) * vol;
    my += 24.0 * (fr.zd[1] + (double)o[1]) * vol;
    mz += 24.0 * (fr.zd[2] + (double)o[2]) * vol;
    bad = __any_sync(FULLMASK, bad);
    st = __reduce_or_sync(FULLMASK, st);
    const double mm[3] = {mx * (1.0 / 24.0), my * (1.0 / 24.0), mz * (1.0 / 24.0)};
    const bool valid = vol > 0.0 && isfinite(vol);
    if (valid) {
        // the centroid is kept in FP32 (frame anchor): one FP32 division per axis
        const float fv = (float)vol;
        for (int a = 0; a < 3; a++) cen[a] = (float)mm[a] / fv;
    }
    if (lane == 0) {
        const double a3 = cp.a * cp.a * cp.a;
        const double a4 = a3 * cp.a;
        cp.vol[i] = vol * a3;
        cp.m1[3 * i + 0] = mm[0] * a4;
        cp.m1[3 * i + 1] = mm[1] * a4;
        cp.m1[3 * i + 2] = mm[2] * a4;
        cp.fcnt[i] = total > FCAP ? FCAP : total;
        cp.topo_n[i] = (uint8_t)(tok && valid ? nt : 0);
        if (valid) {
            cp.anchor[3 * i + 0] = cen[0];
            cp.anchor[3 * i + 1] = cen[1];
            cp.anchor[3 * i + 2] = cen[2];
        }
    }
    return valid;
}

// The cell must stay inside the minimum-image range of every other seed: radius R0 of
// the polytope about the seed against half the box.
template <typename R, class C>
__device__ __noinline__ bool cell_too_large(const Poly<R, C>& P, const CellCtx& cc,
                                            float psimax_glob, float halfLmin, int lane) {
    float r2 = 0.f;
    for (int s = lane; s < P.nt; s += 32) {
        const float dx = (float)P.vx[s] + cc.fr.z[0], dy = (float)P.vy[s] + cc.fr.z[1],
                    dz = (float)P.vz[s] + cc.fr.z[2];
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
    }
    const float R0 = sqrtf(warp_max(r2));
    const float dpsi = fmaxf(psimax_glob - cc.si.phi, 0.f);
    return R0 + sqrtf(R0 * R0 + 2.f * dpsi) > halfLmin * 0.9999f;
}

// An FP32 cell whose centroid lies more than this many spacings from its frame
// origin is clipped once more in a frame at the centroid (its rounding grows with the
// distance of its vertices from the origin)
constexpr float REFRAME_DIST = 0.5f;

// Clip by a list of seeds (warp-uniform count): each lane builds one plane, then the
// warp clips by them in order; entries out of range and seeds already among the
// planes are skipped.
template <typename R, class C>
__device__ __noinline__ int clip_list(Poly<R, C>& P, const ClipParams& cp, const CellCtx& cc,
                                      const int32_t* list, int n, int lane, bool& bad) {
    for (int t0 = 0; t0 < n; t0 += 32) {
        const int t = t0 + lane;
        V4<R> pl;
        pl.x = pl.y = pl.z = pl.w = R(0);
        R len = R(1);
        int32_t j = -1;
        if (t < n) {
            j = list[t];
            if (j >= 0 && j < cp.N && j != (int32_t)cc.i) build_plane(cp, cc, j, pl, len);
            else j = -1;
        }
        const int nk = min(32, n - t0);
        for (int u = 0; u < nk; u++) {
            const int32_t ju = __shfl_sync(FULLMASK, j, u);
            if (ju < 0) continue;
            const V4<R> pn = shfl_plane(pl, u);
            const R plen = __shfl_sync(FULLMASK, len, u);
            if (has_plane(P, ju, lane)) continue;
            const int rc = poly_clip(P, pn, plen, ju, lane, bad);
            if (rc == CLIP_EMPTY || rc == CLIP_CAP) return rc;
        }
    }
    return CLIP_NONE;
}

// Warm start from the cell's stored topology: the planes of its previous facets (and
// the box planes) are rebuilt at the current psi and every stored vertex is
// recomputed from its three planes. The result is the polytope itself when every
// triple is well conditioned and every vertex lies inside every facet plane: the
// stored triangles form a closed surface whose faces lie on bounding planes of the
// intersection, hence its whole boundary. (Box planes need no check: a vertex beyond
// one is more than half a box from its seed, which the size check reports.) Returns
// false when the check fails; the caller then clips from the box.
template <typename R, class C>
__device__ __noinline__ bool topo_init(Poly<R, C>& P, const ClipParams& cp, const CellCtx& cc,
                                       int nf, int nt, int lane) {
    if (6 + nf > C::MP || nt > C::MT || nt > TOPO || nt < 4) return false;
    poly_init(P, cp, cc.fr.z, lane);  // the box planes in slots 0..5
    bool ok = true;
#pragma unroll 1
    for (int k = lane; k < nf; k += 32) {
        const int32_t j = cp.fcol[cc.i * FCAP + k];
        V4<R> pn;
        pn.x = pn.y = pn.z = pn.w = R(0);
        R len = R(1);
        if (j >= 0 && j < cp.N && j != (int32_t)cc.i) build_plane(cp, cc, j, pn, len);
        else ok = false;
        P.pl[6 + k] = pn;
        P.plen[6 + k] = len;
        P.pj[6 + k] = j;
    }
    __syncwarp();
    const R dtol = sizeof(R) == 4 ? R(1e-3) : R(1e-6);
    const uint32_t npl = (uint32_t)(6 + nf);
#pragma unroll 1
    for (int s = lane; s < nt; s += 32) {
        const uint32_t t = cp.topo[cc.i * TOPO + s];
        const uint32_t a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
        if (a >= npl || b >= npl || c >= npl) {
            ok = false;
            continue;
        }
        bool well;
        const V3<R> v = vertex_of(P, t, dtol, well);
        if (!well || !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) ok = false;
        P.tri[s] = t;
        set_vert(P, s, v);
    }
    ok = __all_sync(FULLMASK, ok);
    if (!ok) return false;
#pragma unroll 1
    for (int s = lane; s < nt; s += 32) {
        const V3<R> v = vert(P, s);
        const uint32_t t = P.tri[s];
        const uint32_t a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
        for (uint32_t q = 6; q < npl; q++) {
            if (q == a || q == b || q == c) continue;
            R sd;
            if (beyond(v, P.pl[q], P.plen[q], sd)) ok = false;
        }
    }
    ok = __all_sync(FULLMASK, ok);
    if (lane == 0) {
        P.np = (int)npl;
        P.nt = nt;
    }
    __syncwarp();
    return ok;
}

// global upper bound of psi/a^2 (top pyramid level), every lane
__device__ __forceinline__ float top_psimax(const ClipParams& cp, int lane) {
    float m = -INFINITY;
    const int tl = cp.pyr.nlev - 1;
    const int ntop = cp.pyr.dim[tl][0] * cp.pyr.dim[tl][1] * cp.pyr.dim[tl][2];
    for (int t = lane; t < ntop; t += 32) m = fmaxf(m, cp.pyr.psimax[cp.pyr.off[tl] + t]);
    return warp_max(m);
}

// The cell's carried certificate against its warm-started polytope (bounds b): true when
// it still certifies the cell (see CERT_EPS above). The reserves it used are then written
// back, less the change of psi differences of this evaluation.
template <typename R, class C>
__device__ __noinline__ bool cert_check(Poly<R, C>& P, const ClipParams& cp, const CellCtx& cc,
                                        const Bounds& b, int64_t i, int nc, int lane) {
    const float* cf = cp.cert_f + i * CERT_F;
    const float c0 = cf[0], c1 = cf[1], c2 = cf[2], Rt = cf[3], Mr = cf[4], Wr = cf[5];
    const float hi = ord2f(cp.cert_dpsi[0]), lo = ord2f(cp.cert_dpsi[1]);
    const float cons = __fadd_ru(__fsub_ru(hi, lo), 1e-6f);
    const float Mn = __fsub_rd(Mr, cons), Wn = __fsub_rd(Wr, cons);
    bool ok = nc <= CERT_NEAR && cons >= 0.f && Wn >= 0.f && b.Mv <= Mn;
    // below the stored supports (lane k: direction k)
    if (lane < 27 && lane != 13) {
        const float S = __half2float(__ushort_as_half(cp.cert_s[i * CERT_S + lane]));
        if (!(P.sup[lane] <= S - 1e-5f)) ok = false;
    }
    // inside the stored ball
    float r2 = 0.f;
#pragma unroll 1
    for (int s = lane; s < P.nt; s += 32) {
        const float dx = ((float)P.vx[s] + b.zf[0]) - c0;
        const float dy = ((float)P.vy[s] + b.zf[1]) - c1;
        const float dz = ((float)P.vz[s] + b.zf[2]) - c2;
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
    }
    r2 = warp_max(r2);
    if (!(sqrtf(r2) * (1.f + 1e-6f) + 1e-5f <= Rt)) ok = false;
    if (!__all_sync(FULLMASK, ok)) return false;
    // the recorded seeds, tested exactly as the walk tests a candidate
    V4<R> pl;
    pl.x = pl.y = pl.z = pl.w = R(0);
    R len = R(1);
    const bool have = lane < nc;
    if (have) {
        const int32_t j = cp.cert_j[i * CERT_NEAR + lane];
        if (j >= 0 && j < cp.N && j != (int32_t)cc.i) build_plane(cp, cc, j, pl, len);
        else ok = false;
    }
    if (!__all_sync(FULLMASK, ok)) return false;
    for (uint32_t m = __ballot_sync(FULLMASK, have); m;) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const V4<R> pn = shfl_plane(pl, src);
        const R plen = __shfl_sync(FULLMASK, len, src);
        if (poly_cut_by(P, pn, plen, lane)) return false;
    }
    if (lane == 0) {
        cp.cert_f[i * CERT_F + 4] = Mn;
        cp.cert_f[i * CERT_F + 5] = Wn;
    }
    return true;
}

// Record the certificate of a certifying walk (bounds b before the walk, the seeds in
// P.ftri); its count is set once the cell's outputs are known to be clean.
template <typename R, class C>
__device__ __noinline__ void cert_store(const Poly<R, C>& P, const ClipParams& cp, const Bounds& b,
                                        int64_t i, int lane) {
    if (lane < 27)
        cp.cert_s[i * CERT_S + lane] =
            lane == 13 ? (uint16_t)0 : __half_as_ushort(__float2half_ru(__fadd_ru(P.sup[lane], CERT_EPS)));
    const int n = P.ncert;
    if (lane < n) cp.cert_j[i * CERT_NEAR + lane] = (int32_t)P.ftri[lane];
    if (lane == 0) {
        float* cf = cp.cert_f + i * CERT_F;
        cf[0] = b.c[0];
        cf[1] = b.c[1];
        cf[2] = b.c[2];
        cf[3] = __fadd_ru(b.Rc, CERT_EPS);
        cf[4] = __fadd_ru(b.Mv, CERT_ETA);
        cf[5] = CERT_ETA;
    }
}

// One work item w of a clipping pass: cell worklist[w] (or w), clipped by its first
// candidates, certified (pass 1) or walked (re-queue pass), integrated; outputs
// written, the cell queued for the next pass where needed. BIG: the large-capacity
// FP64 re-clip, after which no pass follows.
template <typename R, class C, int MODE>
__device__ __forceinline__ bool process_cell(Poly<R, C>& P, const ClipParams& cp, int64_t w,
                                             float psimax_glob, float halfLmin, int lane) {
    constexpr bool BIG = C::MP > CapS::MP;
    CellCtx cc;
    cc.i = cp.worklist ? cp.worklist[w] : w;
    const int64_t i = cc.i;
    cc.yi = cp.pos[i];
    cc.psii = cp.psi[i];
    cc.si = load_seed(cp, i);
    bool bad = false;
    uint32_t st = 0;
    float zprev[3] = {cp.anchor[3 * i], cp.anchor[3 * i + 1], cp.anchor[3 * i + 2]};
    if (!(isfinite(zprev[0]) && isfinite(zprev[1]) && isfinite(zprev[2])))
        zprev[0] = zprev[1] = zprev[2] = 0.f;
    // FP32 cells: frame at the previous centroid; FP64 cells: at the seed
    cc.fr = sizeof(R) == 4 ? make_frame(cp, zprev) : seed_frame();
#ifdef SDOT_COUNTERS
    if (lane < 8) P.wc[lane] = 0;
    __syncwarp();
    WCOUNT(P, 6, 1);
#endif
    // first candidates: the cell's facets in the previous diagram (its stored
    // topology when that still holds), then its k nearest seeds (every cell of the
    // first diagram, and any cell without facets)
    int rc = CLIP_NONE;
    const int nprev = cp.facets_valid ? min(cp.fcnt[i], FCAP) : 0;
    const int ntopo = cp.facets_valid ? (int)cp.topo_n[i] : 0;
    bool warm = false;
    if (nprev > 0 && ntopo > 0) warm = topo_init(P, cp, cc, nprev, ntopo, lane);
    if (!warm) {
        poly_init(P, cp, cc.fr.z, lane);
        if (nprev > 0) rc = clip_list(P, cp, cc, cp.fcol + i * FCAP, nprev, lane, bad);
        if (nprev == 0 && rc == CLIP_NONE)
            rc = clip_list(P, cp, cc, cp.knn + i * cp.k, cp.k, lane, bad);
    }
    if (rc == CLIP_EMPTY) st |= CS_EMPTY;
    if (rc == CLIP_CAP) st |= CS_CAPACITY | CS_CAP_POLY;
    // a certifying first pass carries the cell's security certificate between
    // evaluations (see CERT_EPS): used when it still holds, recorded after a walk
    const bool rec = MODE == MODE_CERTIFY && cp.pass == 1 && cp.cert_use;
    // the FP64 re-clip of a cell the FP32 check sent there uses the certificate the
    // first pass kept for it, checked against the FP64 polytope
    const bool use3 = MODE == MODE_FULL && !BIG && cp.pass == 3 && cp.cert_use;
    bool carried = false, stored = false, reframed = false;
    int ncert = -1;
    if (!st) {
        Bounds b;
        for (int a = 0; a < 3; a++) {
            b.yabs[a] = (float)cc.si.c[a] * cp.ht[a] + cc.si.off[a];
            b.zf[a] = cc.fr.z[a];
        }
        b.psi_i = cc.si.phi;
        poly_bounds(P, cp, b, lane);
        if ((rec || use3) && warm) {
            const int nc = cp.cert_n[i];
            if (nc != 0xff) carried = cert_check(P, cp, cc, b, i, nc, lane);
        }
        bool done = true;
        if (!carried) {
            if (rec) {
                if (lane == 0) P.ncert = 0;
                __syncwarp();
            }
            // near-first rings for cells clipped from a list; a warm-started cell of the
            // FP64 re-clip already holds the FP32 pass's polytope, and the pyramid walk
            // below clips every seed that cuts whatever the order
            if (MODE == MODE_FULL && !(warm && cp.pass == 3))
                done = ring_walk(P, cp, cc, b, zprev, lane, bad, st);
            if (done) done = traverse<R, C, MODE>(P, cp, cc, b, lane, bad, st);
            if (done && rec) {
                __syncwarp();
                ncert = P.ncert;
                if (ncert >= 0) {
                    cert_store(P, cp, b, i, lane);
                    stored = true;
                }
            }
        }
        if (!done && MODE == MODE_CERTIFY && (st & CS_UNCERTIFIED)) {
#ifdef SDOT_COUNTERS
            __syncwarp();
            if (lane < 8) atomicAdd(&cp.counters64[lane], (unsigned long long)P.wc[lane]);
            __syncwarp();
#endif
            if (lane == 0) {
                const int32_t q = atomicAdd(cp.queue_cnt, 1);
                cp.queue_out[q] = (int32_t)i;
                cp.status[i] = (uint8_t)st;
                cp.cert_n[i] = 0xff;
            }
            return false;
        }
    }
#ifdef SDOT_COUNTERS
    __syncwarp();
    if (lane < 8) atomicAdd(&cp.counters64[lane], (unsigned long long)P.wc[lane]);
    __syncwarp();
#endif
    if (!st && cell_too_large(P, cc, psimax_glob, halfLmin, lane)) st |= CS_TOO_LARGE;
    float cen[3];
    bool have_cen = false;
    if (!(st & (CS_EMPTY | CS_CAPACITY)))
        have_cen = integrate(P, cp, cc.fr, i, lane, bad, st, cen);
    // FP32 cells far from their frame origin (the first diagram of a context, or a
    // large step of psi): clip again by the facets just found, in a frame at the
    // centroid just found. The facets are the cell's complete neighbour set, so no
    // walk is needed; the outputs are overwritten.
    if (sizeof(R) == 4 && have_cen && !(st & (CS_EMPTY | CS_CAPACITY | CS_TOO_LARGE))) {
        float dz2 = 0.f;
#pragma unroll
        for (int a = 0; a < 3; a++) dz2 += (cen[a] - cc.fr.z[a]) * (cen[a] - cc.fr.z[a]);
        if (dz2 > REFRAME_DIST * REFRAME_DIST) {
            reframed = true;
            __syncwarp();  // facets and counts written by integrate
            const int nf = min(cp.fcnt[i], FCAP);
            __syncwarp();
            cc.fr = make_frame(cp, cen);
            bad = false;
            st = 0;
            poly_init(P, cp, cc.fr.z, lane);
            const int rc2 = clip_list(P, cp, cc, cp.fcol + i * FCAP, nf, lane, bad);
            if (rc2 == CLIP_EMPTY) st |= CS_EMPTY;
            if (rc2 == CLIP_CAP) st |= CS_CAPACITY | CS_CAP_POLY;
            if (!st && cell_too_large(P, cc, psimax_glob, halfLmin, lane)) st |= CS_TOO_LARGE;
            if (!(st & (CS_EMPTY | CS_CAPACITY))) integrate(P, cp, cc.fr, i, lane, bad, st, cen);
        }
    }
    if (bad) st |= CS_INCONSISTENT;
    if (lane == 0) {
        if (st & (CS_EMPTY | CS_CAPACITY)) {
            // no facets from this cell (an empty cell has none; a cell over capacity
            // is re-clipped or reported, and must not leave stale facet counts)
            cp.fcnt[i] = 0;
        }
        if (st & CS_EMPTY) {
            cp.vol[i] = 0.0;
            cp.m1[3 * i] = cp.m1[3 * i + 1] = cp.m1[3 * i + 2] = 0.0;
        }
        // FP32 cells failing a check, and cells over the small capacity, are clipped
        // again in FP64 (small polytope first, the large one for its overflows)
        const bool redo = !BIG && (((sizeof(R) == 4) && (st & CS_INCONSISTENT)) ||
                                   (st & CS_CAPACITY));
        // the topology stays only where it is whole: an FP32 cell sent to the FP64
        // re-clip keeps it as that pass's warm start, which validates it in FP64
        const bool keep_topo =
            !(st & (CS_EMPTY | CS_CAPACITY)) &&
            (!(st & CS_INCONSISTENT) || (redo && (st & CS_INCONSISTENT) == st));
        if (!keep_topo) cp.topo_n[i] = 0;
        // history of the evaluation kept in the final status: a cell of the re-queue
        // pass was re-queued (8); a cell of the FP64 re-clip keeps what sent it there
        // (4: FP32 check failed, 32/64/128: small capacity exceeded) and its re-queue
        uint32_t hist = 0;
        if (cp.pass == 2) hist = CS_UNCERTIFIED;
        if (cp.pass == 3)
            hist = cp.status[i] & (CS_INCONSISTENT | CS_UNCERTIFIED | CS_CAP_POLY | CS_CAP_FACE |
                                   CS_CAP_STACK);
        cp.status[i] = (uint8_t)(st | hist);
        if (redo) {
            const int32_t q = atomicAdd(cp.q64_cnt, 1);
            cp.q64_out[q] = (int32_t)i;
        }
        // the certificate stays valid only for a clean cell whose every plane other
        // than the box's is a facet (the planes of its next warm start); a first-pass
        // cell whose only failure is the FP32 check keeps it for its FP64 re-clip
        const bool facets = !reframed && cp.fcnt[i] == P.np - 6;
        const bool keep1 = rec && facets && (carried || stored) &&
                           (st == 0 || (redo && st == CS_INCONSISTENT));
        const bool keep3 = use3 && facets && carried && st == 0;
        if (!(keep1 || keep3)) cp.cert_n[i] = 0xff;
        else if (keep1 && stored) cp.cert_n[i] = (uint8_t)ncert;
    }
    return rec && carried;
}

}  // namespace sdot

namespace sdot {

// Volume of the polytope (units of a^3), FP64 sum of per-face fan tetrahedra from the
// centre of the vertices' bounding box, the faces found as in integrate. Every lane
// gets the value; 0 when a face cycle is broken.
template <typename R, class C>
__device__ __noinline__ double poly_volume(Poly<R, C>& P, int lane) {
    constexpr int FPL = (C::MP + 31) / 32;
    R o[3];
    {
        R mn[3] = {R(1e30), R(1e30), R(1e30)}, mxv[3] = {R(-1e30), R(-1e30), R(-1e30)};
        for (int s2 = lane; s2 < P.nt; s2 += 32) {
            const R v[3] = {P.vx[s2], P.vy[s2], P.vz[s2]};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                mn[a] = fmin(mn[a], v[a]);
                mxv[a] = fmax(mxv[a], v[a]);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
            for (int q = 16; q > 0; q >>= 1) {
                mn[a] = fmin(mn[a], __shfl_xor_sync(FULLMASK, mn[a], q));
                mxv[a] = fmax(mxv[a], __shfl_xor_sync(FULLMASK, mxv[a], q));
            }
            o[a] = R(0.5) * (mn[a] + mxv[a]);
        }
    }
    const int nt = P.nt, np = P.np;
    for (int f = lane; f < np; f += 32) P.fend[f] = 0u;
    __syncwarp();
    for (int s2 = lane; s2 < nt; s2 += 32) {
        const uint32_t t = P.tri[s2];
        atomicAdd(&P.fend[t & 0xff], 1u);
        atomicAdd(&P.fend[(t >> 8) & 0xff], 1u);
        atomicAdd(&P.fend[(t >> 16) & 0xff], 1u);
    }
    __syncwarp();
    int fcount[FPL];
    {
        uint32_t carry = 0;
        for (int k = 0; k < FPL; k++) {
            const int f = lane + 32 * k;
            const uint32_t c = f < np ? P.fend[f] : 0u;
            fcount[k] = (int)c;
            uint32_t incl = c;
            for (int q = 1; q < 32; q <<= 1) {
                const uint32_t y = __shfl_up_sync(FULLMASK, incl, q);
                if (lane >= q) incl += y;
            }
            if (f < np) P.fend[f] = carry + incl - c;
            carry += __shfl_sync(FULLMASK, incl, 31);
        }
    }
    __syncwarp();
    for (int s2 = lane; s2 < nt; s2 += 32) {
        const uint32_t t = P.tri[s2];
        const uint32_t a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
        const uint32_t sv = (uint32_t)s2 << 16;
        P.fent[atomicAdd(&P.fend[a], 1u)] = b | (c << 8) | sv;
        P.fent[atomicAdd(&P.fend[b], 1u)] = c | (a << 8) | sv;
        P.fent[atomicAdd(&P.fend[c], 1u)] = a | (b << 8) | sv;
    }
    __syncwarp();
    double vol6 = 0.0;
    bool ok = true;
    for (int k = 0; k < FPL; k++) {
        const int f = lane + 32 * k;
        const int m = fcount[k];
        if (f >= np || m == 0) continue;
        if (m < 3) {
            ok = false;
            continue;
        }
        const int e0 = (int)P.fend[f] - m;
        int first = e0;
        for (int e = e0 + 1; e < e0 + m; e++)
            if ((P.fent[e] >> 16) < (P.fent[first] >> 16)) first = e;
        uint32_t ecur = P.fent[first];
        const uint32_t x0 = ecur & 0xff;
        V3<R> v0 = vert(P, ecur >> 16);
        v0.x -= o[0];
        v0.y -= o[1];
        v0.z -= o[2];
        V3<R> vp = v0;
        R fv6 = 0;
        for (int step = 1; step < m; step++) {
            const uint32_t yv = (ecur >> 8) & 0xff;
            int nxt = -1;
            for (int e = e0; e < e0 + m; e++)
                if ((P.fent[e] & 0xff) == yv) {
                    nxt = e;
                    break;
                }
            if (nxt < 0 || nxt == first) {
                ok = false;
                break;
            }
            ecur = P.fent[nxt];
            V3<R> vc = vert(P, ecur >> 16);
            vc.x -= o[0];
            vc.y -= o[1];
            vc.z -= o[2];
            if (step >= 2) {
                const R ax = vp.x - v0.x, ay = vp.y - v0.y, az = vp.z - v0.z;
                const R bx = vc.x - v0.x, by = vc.y - v0.y, bz = vc.z - v0.z;
                const R cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
                fv6 += v0.x * cx + v0.y * cy + v0.z * cz;
            }
            vp = vc;
        }
        if (((ecur >> 8) & 0xff) != x0) ok = false;
        vol6 += (double)fv6;
    }
    vol6 = warp_sum(vol6);
    ok = __all_sync(FULLMASK, ok);
    return ok ? vol6 / 6.0 : 0.0;
}

// P2 <- P1 (warp-uniform)
template <typename R, class C>
__device__ __noinline__ void poly_copy(Poly<R, C>& P2, const Poly<R, C>& P1, int lane) {
    for (int q = lane; q < P1.np; q += 32) {
        P2.pl[q] = P1.pl[q];
        P2.plen[q] = P1.plen[q];
        P2.pj[q] = P1.pj[q];
    }
    for (int s = lane; s < P1.nt; s += 32) {
        P2.tri[s] = P1.tri[s];
        P2.vx[s] = P1.vx[s];
        P2.vy[s] = P1.vy[s];
        P2.vz[s] = P1.vz[s];
    }
    if (lane == 0) {
        P2.np = P1.np;
        P2.nt = P1.nt;
    }
    __syncwarp();
}

}  // namespace sdot
