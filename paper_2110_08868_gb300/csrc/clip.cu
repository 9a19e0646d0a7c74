// Laguerre cell clipping: volumes, first moments and facet areas of every cell.
//
// Cell i of eq. (laguerrecell) in seed-local coordinates p = q - y_i is
//     P_i = { p : p.d_ij <= b_ij for all j },  d_ij = minimum image of y_j - y_i,
//     b_ij = 1/2 |d_ij|^2 + psi_i - psi_j,
// the lifted power bisectors of the neighbours. Coordinates are scaled by the
// length unit a = (|box|/N)^(1/3) and psi by a^2 so every quantity is O(1).
//
// One warp owns one cell. The polytope lives in shared memory as planes plus its
// vertices, each vertex a "dual triangle" of the three planes through it, oriented
// so that det(n_a, n_b, n_c) > 0. Clipping by a new plane: the lanes classify the
// vertices (one ballot), the removed vertices' dual edges whose reverse edge is
// not removed form the boundary cycle, and every boundary edge (a -> b) yields the
// new vertex (a, b, new plane). Integration walks each face's vertex cycle and
// sums fan tetrahedra from the centre of the vertices' bounding box (volume,
// first moment, area vector).
//
// Neighbour search: the k nearest seeds first, then a security test. The test
// walks a pyramid of per-node upper bounds of psi and proves, node by node, that no
// other seed's plane can reach the polytope:
//     seed j cannot cut if  z.d + R_z |d| <= b_ij
// for any anchor z with R_z = max_vertex |v - z| (z: the cell's previous local
// centroid). For a node B with distance u from the anchor, distance at most dmax
// from the seed and psi bound psimax_B this holds for every seed inside when
//     1/2 u^2 - 1/2 |z|^2 - R_z dmax - (psimax_B - psi_i) >= 0.
// A cell whose test finds a seed that actually cuts it is re-queued; the re-queue
// pass clips every such seed during the same walk. In mixed precision the geometry
// runs in FP32 and cells failing the consistency check (non-closed surface, broken
// face cycle, badly conditioned vertex, capacity) are re-clipped in FP64. The FP32
// polytope is held relative to a frame origin z near the cell (its previous
// centroid), where the bisector of seed j reads
//     q.d_ij <= b_ij - d_ij.z,   p = z + q,
// with the offset summed in FP64 from the exact seed difference: a cell far from its
// own seed (pushed away by a clump) keeps vertex coordinates and plane offsets of
// its own size, so FP32 rounding is relative to the cell, not to its distance from
// the seed. Sums are accumulated in FP64.
#include <float.h>
#include <math.h>

#include <string>
#include <vector>

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

template <typename R>
struct WarpPoly {
    V4<R> pl[MAXP];         // plane p.n <= w, n = d/a, w = b/a^2
    R plen[MAXP];           // |n|
    int32_t pj[MAXP];       // neighbour (sorted index) or -1 for a box face
    uint32_t tri[MAXT];     // plane slots a | b << 8 | c << 16
    V3<R> v[MAXT];          // vertex positions
    uint32_t scratch[MAXT]; // removed vertices during a clip
    uint32_t fresh[MAXT];   // new vertices during a clip
    V3<R> freshv[MAXT];     // their positions
    uint32_t stack[STACK];  // traversal stack: level << 27 | node
    int np, nt;
    uint32_t wc[8];         // work counters of the current cell (diagnostic builds)
};

// Work counters, compiled in only with -DSDOT_COUNTERS (diagnostic builds). The
// count argument is evaluated by lane 0 only, so it must not contain a warp vote:
// take votes before the macro.
// 0 clip calls, 1 cuts, 2 node tests, 3 leaf visits, 4 seed tests, 5 candidates,
// 6 cells, 7 pyramid-walk rounds
#ifdef SDOT_COUNTERS
#define WCOUNT(P, k, n)                 \
    do {                                \
        if ((threadIdx.x & 31) == 0) (P).wc[k] += (n); \
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
__device__ __forceinline__ double exact_d2(const Pos4& a, const Pos4& b,
                                           const ClipParams& p) {
    double dx = wrapd(__dsub_rn(b.x, a.x), p.L[0], p.halfL[0]);
    double dy = wrapd(__dsub_rn(b.y, a.y), p.L[1], p.halfL[1]);
    double dz = wrapd(__dsub_rn(b.z, a.z), p.L[2], p.halfL[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ uint32_t pack3(uint32_t a, uint32_t b, uint32_t c) {
    return a | (b << 8) | (c << 16);
}
__device__ __forceinline__ bool has_edge(uint32_t t, uint32_t x, uint32_t y) {
    // does triangle t contain the directed edge x -> y
    uint32_t a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
    return (a == x && b == y) || (b == x && c == y) || (c == x && a == y);
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

// the box [-L/2, L/2]^3: bisectors with the seed's own six face images
// The periodic box around the seed: the bisectors of the cell's own images at
// +-Lt e_a, written relative to the frame origin z (zero: the seed itself).
template <typename R>
__device__ void poly_init(WarpPoly<R>& P, const ClipParams& cp, const float* z, int lane) {
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
        V3<R> v;
        v.x = R(0.5) * (R)cp.Lt[0] * (R)sx - (R)z[0];
        v.y = R(0.5) * (R)cp.Lt[1] * (R)sy - (R)z[1];
        v.z = R(0.5) * (R)cp.Lt[2] * (R)sz - (R)z[2];
        P.v[lane] = v;
    }
    if (lane == 0) {
        P.np = 6;
        P.nt = 8;
    }
    __syncwarp();
}

template <typename R>
__device__ __forceinline__ V3<R> vertex_of(const WarpPoly<R>& P, uint32_t t, R& det_rel) {
    const V4<R> A = P.pl[t & 0xff], B = P.pl[(t >> 8) & 0xff], C = P.pl[(t >> 16) & 0xff];
    // n_b x n_c, n_c x n_a, n_a x n_b
    R bcx = B.y * C.z - B.z * C.y, bcy = B.z * C.x - B.x * C.z, bcz = B.x * C.y - B.y * C.x;
    R cax = C.y * A.z - C.z * A.y, cay = C.z * A.x - C.x * A.z, caz = C.x * A.y - C.y * A.x;
    R abx = A.y * B.z - A.z * B.y, aby = A.z * B.x - A.x * B.z, abz = A.x * B.y - A.y * B.x;
    R det = A.x * bcx + A.y * bcy + A.z * bcz;
    R inv = R(1) / det;
    V3<R> v;
    v.x = (A.w * bcx + B.w * cax + C.w * abx) * inv;
    v.y = (A.w * bcy + B.w * cay + C.w * aby) * inv;
    v.z = (A.w * bcz + B.w * caz + C.w * abz) * inv;
    R la = P.plen[t & 0xff], lb = P.plen[(t >> 8) & 0xff], lc = P.plen[(t >> 16) & 0xff];
    det_rel = det / (la * lb * lc);
    return v;
}

// drop planes no vertex references any more; returns the number of planes left
template <typename R>
__device__ __noinline__ int poly_gc(WarpPoly<R>& P, int lane) {
    constexpr int NW = MAXP / 32;
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
    const uint32_t below = (lane == 0) ? 0u : ((1u << lane) - 1u);
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

// Clip by p.n <= w (tag j). Non-finite geometry sets bad.
template <typename R>
__device__ __forceinline__ int poly_clip_inl(WarpPoly<R>& P, const V4<R>& pn, R plen, int32_t j,
                                             int lane, bool& bad) {
    constexpr int SL = MAXT / 32;  // vertex slots per lane
    const int nt = P.nt;
    bool out[SL];
    uint32_t m[SL];
    int nrem = 0;
#pragma unroll
    for (int t = 0; t < SL; t++) {
        int s = lane + 32 * t;
        out[t] = false;
        m[t] = 0u;
        if (32 * t < nt) {  // warp-uniform
            if (s < nt) {
                R sd;
                out[t] = beyond(P.v[s], pn, plen, sd);
            }
            m[t] = __ballot_sync(FULLMASK, out[t]);
            nrem += __popc(m[t]);
        }
    }
    WCOUNT(P, 0, 1);
    if (nrem == 0) return CLIP_NONE;
    WCOUNT(P, 1, 1);
    if (nrem == nt) return CLIP_EMPTY;
    if (P.np >= MAXP) {
        if (poly_gc(P, lane) >= MAXP) return CLIP_CAP;
    }
    const uint32_t ps = (uint32_t)P.np;
    const uint32_t below = (lane == 0) ? 0u : ((1u << lane) - 1u);
    // removed list: triangle | slot << 24
    {
        int base = 0;
#pragma unroll
        for (int t = 0; t < SL; t++) {
            if (out[t]) P.scratch[base + __popc(m[t] & below)] =
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
        uint32_t t = P.scratch[r] & 0xffffffu;
        uint32_t a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
        bool fab = false, fbc = false, fca = false;
        for (int q = 0; q < nrem; q++) {
            uint32_t u = P.scratch[q] & 0xffffffu;
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
    if (nkept + nnew > MAXT) return CLIP_CAP;
    // new vertices: the plane through the edge's two planes and the new plane; when
    // that system is ill-conditioned (the new plane almost parallel to the edge) the
    // vertex is interpolated on the edge between its kept and removed end points
    bool lbad = false;
    {
        int pos = incl - cnt;
        const R dtol = sizeof(R) == 4 ? R(1e-3) : R(1e-6);
        for (int r = lane, e = 0; r < nrem; r += 32, e++) {
            uint32_t rr = P.scratch[r];
            uint32_t t = rr & 0xffffffu, sr = rr >> 24;
            uint32_t tv[3] = {t & 0xff, (t >> 8) & 0xff, (t >> 16) & 0xff};
            uint32_t bits = (bmask >> (3 * e)) & 7u;
            for (int k = 0; k < 3; k++) {
                if (!(bits >> k & 1u)) continue;
                uint32_t x = tv[k], y = tv[(k + 1) % 3];
                uint32_t nt3 = pack3(x, y, ps);
                R det_rel;
                V3<R> v = vertex_of(P, nt3, det_rel);
                if (!(det_rel > dtol)) {
                    int sk = -1;
                    for (int q = 0; q < nt; q++) {
                        bool o = (m[q >> 5] >> (q & 31)) & 1u;
                        if (!o && has_edge(P.tri[q], y, x)) { sk = q; break; }
                    }
                    if (sk >= 0) {
                        V3<R> vk = P.v[sk], vr = P.v[sr];
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
                P.fresh[pos] = nt3;
                P.freshv[pos] = v;
                pos++;
            }
        }
    }
    __syncwarp();
    // compact the kept vertices (read all, then write)
    {
        uint32_t kt[SL];
        V3<R> kv[SL];
        int dst[SL];
        int base = 0;
#pragma unroll
        for (int t = 0; t < SL; t++) {
            int s = lane + 32 * t;
            dst[t] = -1;
            if (32 * t < nt) {  // warp-uniform
                bool keep = s < nt && !out[t];
                uint32_t km = __ballot_sync(FULLMASK, keep);
                if (keep) {
                    kt[t] = P.tri[s];
                    kv[t] = P.v[s];
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
                P.v[dst[t]] = kv[t];
            }
    }
    __syncwarp();
    for (int n = lane; n < nnew; n += 32) {
        P.tri[nkept + n] = P.fresh[n];
        P.v[nkept + n] = P.freshv[n];
    }
    if (lane == 0) {
        P.np = ps + 1;
        P.nt = nkept + nnew;
    }
    if (__any_sync(FULLMASK, lbad)) bad = true;
    __syncwarp();
    return CLIP_CUT;
}

template <typename R>
__device__ __noinline__ int poly_clip(WarpPoly<R>& P, const V4<R>& pn, R plen, int32_t j, int lane,
                                      bool& bad) {
    return poly_clip_inl(P, pn, plen, j, lane, bad);
}

template <typename R>
__device__ R poly_radius(const WarpPoly<R>& P, V3<R> z, int lane) {
    R r2 = 0;
    for (int s = lane; s < P.nt; s += 32) {
        V3<R> v = P.v[s];
        R dx = v.x - z.x, dy = v.y - z.y, dz = v.z - z.z;
        R q = dx * dx + dy * dy + dz * dz;
        r2 = q > r2 ? q : r2;
    }
    r2 = warp_max(r2);
    return sqrt(r2);
}

// plane of neighbour j for cell i, built in FP64 (normalised units)
__device__ __forceinline__ void make_plane(const ClipParams& cp, const Pos4& yi, double psii,
                                           int32_t j, double& nx, double& ny, double& nz,
                                           double& w) {
    Pos4 yj = cp.pos[j];
    nx = wrapd(yj.x - yi.x, cp.L[0], cp.halfL[0]) * cp.inv_a;
    ny = wrapd(yj.y - yi.y, cp.L[1], cp.halfL[1]) * cp.inv_a;
    nz = wrapd(yj.z - yi.z, cp.L[2], cp.halfL[2]) * cp.inv_a;
    w = 0.5 * (nx * nx + ny * ny + nz * nz) + (psii - cp.psi[j]) * cp.inv_a2;
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
    float z[3];   // z in FP32
    double zd[3]; // z in FP64
};

__device__ __forceinline__ Frame make_frame(const ClipParams& cp, const float* zwant) {
    Frame f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float za = zwant[a];
        if (!isfinite(za)) za = 0.f;
        za = fminf(fmaxf(za, -cp.halfLt[a]), cp.halfLt[a]);
        const double q = (double)cp.ht[a] * (1.0 / 4096.0);
        f.zd[a] = (double)llrint((double)za / q) * q;
        f.z[a] = (float)f.zd[a];
    }
    return f;
}

// the frame at the seed itself (FP64 cells, first diagram)
__device__ __forceinline__ Frame seed_frame() {
    Frame f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        f.z[a] = 0.f;
        f.zd[a] = 0.0;
    }
    return f;
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

// FP32 plane of seed j for cell i from grid-local coordinates: the integer part of
// the difference is exact, so the plane is accurate to FP32 relative precision of
// |d| and of the psi difference (psi carried as hi + lo floats).
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

__device__ __forceinline__ float circ_gap(float p, float lo, float hi, float Lt) {
    // distance from p to the interval [lo, hi] on a circle of length Lt
    if (p >= lo && p <= hi) return 0.f;
    float d1 = lo - p;
    if (d1 < 0.f) d1 += Lt;
    float d2 = p - hi;
    if (d2 < 0.f) d2 += Lt;
    return fminf(d1, d2);
}
__device__ __forceinline__ float circ_far(float p, float lo, float hi, float Lt) {
    // largest circular distance from p to a point of [lo, hi]
    float A = p + 0.5f * Lt;
    if (A >= Lt) A -= Lt;
    if (A >= lo && A <= hi) return 0.5f * Lt;
    float e1 = fabsf(lo - p), e2 = fabsf(hi - p);
    e1 = fminf(e1, Lt - e1);
    e2 = fminf(e2, Lt - e2);
    return fmaxf(e1, e2);
}

// Current bounds of the polytope: box [bmin, bmax], its centre c and the radius Rc of
// the smallest ball around c holding every vertex (local coordinates, units of a).
struct Bounds {
    float zf[3];  // frame origin of the polytope's vertices (relative to the seed)
    float bmin[3], bmax[3];
    float c[3];
    float Rc;
    float cabs[3];  // c in absolute coordinates, wrapped into the box
    float yabs[3];  // the seed in absolute coordinates
    float c2h;      // 1/2 |c|^2
    float psi_i;    // psi_i / a^2 (hi part)
};

template <typename R>
__device__ void poly_bounds(const WarpPoly<R>& P, const ClipParams& cp, Bounds& b, int lane) {
    float mn[3] = {1e30f, 1e30f, 1e30f}, mx[3] = {-1e30f, -1e30f, -1e30f};
    for (int s = lane; s < P.nt; s += 32) {
        V3<R> v = P.v[s];
        float vv[3] = {(float)v.x + b.zf[0], (float)v.y + b.zf[1], (float)v.z + b.zf[2]};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            mn[a] = fminf(mn[a], vv[a]);
            mx[a] = fmaxf(mx[a], vv[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(FULLMASK, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(FULLMASK, mx[a], o));
        }
        b.bmin[a] = mn[a];
        b.bmax[a] = mx[a];
        b.c[a] = 0.5f * (mn[a] + mx[a]);
    }
    float r2 = 0.f;
    for (int s = lane; s < P.nt; s += 32) {
        V3<R> v = P.v[s];
        float dx = ((float)v.x + b.zf[0]) - b.c[0], dy = ((float)v.y + b.zf[1]) - b.c[1],
              dz = ((float)v.z + b.zf[2]) - b.c[2];
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
    }
    r2 = warp_max(r2);
    b.Rc = sqrtf(r2) * 1.0001f + 1e-5f;
    b.c2h = 0.5f * (b.c[0] * b.c[0] + b.c[1] * b.c[1] + b.c[2] * b.c[2]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float za = b.yabs[a] + b.c[a];
        za = fmodf(za, cp.Lt[a]);
        if (za < 0.f) za += cp.Lt[a];
        if (za >= cp.Lt[a]) za = 0.f;
        b.cabs[a] = za;
    }
}

// min over d in [l, h] of f(d) = 1/2 d^2 - max(d bmax, d bmin) (a piecewise parabola
// with its minima at d = bmax >= 0 and d = bmin <= 0)
__device__ __forceinline__ float fmin_axis(float l, float h, float bmn, float bmx) {
    float fl = 0.5f * l * l - (l >= 0.f ? l * bmx : l * bmn);
    float fh = 0.5f * h * h - (h >= 0.f ? h * bmx : h * bmn);
    float m = fminf(fl, fh);
    if (bmx > 0.f && l < bmx && bmx < h) m = fminf(m, -0.5f * bmx * bmx);
    if (bmn < 0.f && l < bmn && bmn < h) m = fminf(m, -0.5f * bmn * bmn);
    return m;
}

// True when no seed of node (level l, coordinates X, Y, Z) can cut the polytope. For a
// seed j with d = its minimum-image offset, max_vertex v.d <= S(d) = sum_a max(d_a bmax_a,
// d_a bmin_a) (support of the bounding box), so j cannot cut when
//     sum_a [1/2 d_a^2 - max(d_a bmax_a, d_a bmin_a)] >= psi_j - psi_i.
// Each term is minimised over the node's offset interval on its axis, psi_j is bounded
// by the node's psimax.
__device__ __forceinline__ bool node_pruned(const ClipParams& cp, const Bounds& b, int l, int X,
                                            int Y, int Z) {
    float pm = cp.pyr.psimax[cp.pyr.off[l] +
                             ((int64_t)Z * cp.pyr.dim[l][1] + Y) * cp.pyr.dim[l][0] + X];
    if (pm == -INFINITY) return true;  // no seed inside
    int span = 1 << (2 * l);
    int c[3] = {X, Y, Z};
    float val = 0.f, mag = 0.f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int c0 = c[a] * span, c1 = min((c[a] + 1) * span, cp.G[a]);
        float lo = c0 * cp.ht[a], hi = (c1 == cp.G[a]) ? cp.Lt[a] : c1 * cp.ht[a];
        const float Lt = cp.Lt[a], hL = cp.halfLt[a];
        float w = hi - lo;
        float m;
        if (w >= Lt) {
            m = fmin_axis(-hL, hL, b.bmin[a], b.bmax[a]);
        } else {
            float o = lo - b.yabs[a];  // offset of the node start, minimum image
            o -= Lt * floorf((o + hL) / Lt);
            if (o + w <= hL) {
                m = fmin_axis(o, o + w, b.bmin[a], b.bmax[a]);
            } else {  // the interval wraps through +-L/2
                m = fminf(fmin_axis(o, hL, b.bmin[a], b.bmax[a]),
                          fmin_axis(-hL, o + w - Lt, b.bmin[a], b.bmax[a]));
            }
        }
        val += m;
        mag += fabsf(m);
    }
    float dpsi = pm - b.psi_i;
    float margin = 2e-5f * (mag + fabsf(pm) + fabsf(b.psi_i)) + 1e-5f;
    if (val - dpsi > margin) return true;
    // second valid bound, better in diagonal directions: every vertex lies within Rc
    // of the box centre c, so max_v v.d <= c.d + Rc |d|, and 1/2|d|^2 - c.d =
    // 1/2|d - c|^2 - 1/2|c|^2 with |d - c| >= u (anchor-to-node distance), |d| <= dmax
    float u2 = 0.f, dm2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int c0 = c[a] * span, c1 = min((c[a] + 1) * span, cp.G[a]);
        float lo = c0 * cp.ht[a], hi = (c1 == cp.G[a]) ? cp.Lt[a] : c1 * cp.ht[a];
        float g = circ_gap(b.cabs[a], lo, hi, cp.Lt[a]);
        float f = circ_far(b.yabs[a], lo, hi, cp.Lt[a]);
        u2 += g * g;
        dm2 += f * f;
    }
    float t1 = 0.5f * u2, t2 = b.Rc * sqrtf(dm2);
    float val2 = t1 - b.c2h - t2 - dpsi;
    float margin2 = 2e-5f * (t1 + b.c2h + t2 + fabsf(pm) + fabsf(b.psi_i)) + 1e-5f;
    return val2 > margin2;
}

// conservative FP32 test: can the plane (n, w) reach the polytope? Two valid upper
// bounds of max_vertex v.n are used, the support of the bounding box and that of the
// ball of radius Rc around the box centre c; the plane is a candidate only if both
// reach it.
__device__ __forceinline__ bool box_may_cut(const Bounds& b, float nx, float ny, float nz,
                                            float w) {
    float sx = nx > 0.f ? nx * b.bmax[0] : nx * b.bmin[0];
    float sy = ny > 0.f ? ny * b.bmax[1] : ny * b.bmin[1];
    float sz = nz > 0.f ? nz * b.bmax[2] : nz * b.bmin[2];
    float S = sx + sy + sz;
    float margin = 2e-5f * (fabsf(sx) + fabsf(sy) + fabsf(sz) + fabsf(w)) + 1e-5f;
    if (!(S > w - margin)) return false;
    float cn = b.c[0] * nx + b.c[1] * ny + b.c[2] * nz;
    float rn = b.Rc * sqrtf(nx * nx + ny * ny + nz * nz);
    float margin2 = 2e-5f * (fabsf(cn) + rn + fabsf(w)) + 1e-5f;
    return cn + rn > w - margin2;
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

// One candidate seed j (warp-uniform): skip it if it already is a plane of the
// polytope or its plane leaves every vertex inside; otherwise CERTIFY fails and FULL
// clips. Returns LEAF_STOP when the cell's processing must stop.
template <typename R, int MODE>
__device__ int candidate(WarpPoly<R>& P, const ClipParams& cp, const CellCtx& cc, Bounds& b,
                         int32_t j, int lane, bool& bad, uint32_t& st) {
    bool dup = false;
#pragma unroll
    for (int w = 0; w < MAXP / 32; w++)
        dup |= (lane + 32 * w < P.np && P.pj[lane + 32 * w] == j);
    if (__any_sync(FULLMASK, dup)) return LEAF_OK;
    V4<R> pn;
    R plen;
    build_plane(cp, cc, j, pn, plen);
    if (MODE == MODE_CERTIFY) {
        bool o = false;
        for (int q = lane; q < P.nt; q += 32) {
            R sd;
            o |= beyond(P.v[q], pn, plen, sd);
        }
        if (__any_sync(FULLMASK, o)) {
            st |= CS_UNCERTIFIED;
            return LEAF_STOP;
        }
        return LEAF_OK;
    }
    int rc = poly_clip(P, pn, plen, j, lane, bad);
    if (rc == CLIP_EMPTY) {
        st |= CS_EMPTY;
        return LEAF_STOP;
    }
    if (rc == CLIP_CAP) {
        st |= CS_CAPACITY | CS_CAP_POLY;
        return LEAF_STOP;
    }
    if (rc == CLIP_CUT) poly_bounds(P, cp, b, lane);
    return LEAF_OK;
}

// The seeds of up to 32 grid cells at once, one grid cell per lane (leaf < 0: none).
template <typename R, int MODE>
__device__ __noinline__ int process_leaves(WarpPoly<R>& P, const ClipParams& cp,
                                           const CellCtx& cc, Bounds& b, int64_t leaf, int lane,
                                           bool& bad, uint32_t& st) {
    int32_t sb = 0, se = 0;
    if (leaf >= 0) {
        sb = cp.cell_start[leaf];
        se = cp.cell_start[leaf + 1];
    }
    int n = se - sb;
    int maxn = n;
    for (int o = 16; o > 0; o >>= 1) maxn = max(maxn, __shfl_xor_sync(FULLMASK, maxn, o));
#ifdef SDOT_COUNTERS
    {
        const uint32_t nleaf = __popc(__ballot_sync(FULLMASK, leaf >= 0));
        WCOUNT(P, 3, nleaf);
    }
#endif
    for (int u = 0; u < maxn; u++) {
        int32_t s = sb + u;
        bool cand = false;
        if (u < n && s != (int32_t)cc.i) {
            float nx, ny, nz, w;
            plane_f32(cp, cc.si, s, nx, ny, nz, w);
            cand = box_may_cut(b, nx, ny, nz, w);
        }
#ifdef SDOT_COUNTERS
        {
            const uint32_t nseed = __popc(__ballot_sync(FULLMASK, u < n));
            WCOUNT(P, 4, nseed);
        }
#endif
        uint32_t cm = __ballot_sync(FULLMASK, cand);
        WCOUNT(P, 5, __popc(cm));
        while (cm) {
            int src = __ffs(cm) - 1;
            cm &= cm - 1;
            int32_t j = __shfl_sync(FULLMASK, s, src);
            if (candidate<R, MODE>(P, cp, cc, b, j, lane, bad, st) == LEAF_STOP) return LEAF_STOP;
        }
    }
    return LEAF_OK;
}

// Near-first pass for re-queued cells: the grid cells in Chebyshev rings around the
// grid cell of the previous centroid, so the polytope is small before the pyramid
// walk (which visits nodes in no particular order) starts.
template <typename R>
__device__ __noinline__ bool ring_walk(WarpPoly<R>& P, const ClipParams& cp, const CellCtx& cc,
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
            int t = base + lane;
            int64_t leaf = -1;
            if (t < n3) {
                int ox = t % w - r, oy = (t / w) % w - r, oz = t / (w * w) - r;
                int ch = max(abs(ox), max(abs(oy), abs(oz)));
                if (ch == r) {
                    int cx = ((ca[0] + ox) % cp.G[0] + cp.G[0]) % cp.G[0];
                    int cy = ((ca[1] + oy) % cp.G[1] + cp.G[1]) % cp.G[1];
                    int cz = ((ca[2] + oz) % cp.G[2] + cp.G[2]) % cp.G[2];
                    leaf = ((int64_t)cz * cp.G[1] + cy) * cp.G[0] + cx;
                }
            }
            if (process_leaves<R, MODE_FULL>(P, cp, cc, b, leaf, lane, bad, st) == LEAF_STOP)
                return false;
        }
    }
    return true;
}

// Walk the pyramid. MODE_CERTIFY: return false as soon as a seed cuts the polytope.
// MODE_FULL: clip every such seed. Returns true when the walk completed.
template <typename R, int MODE>
__device__ bool traverse(WarpPoly<R>& P, const ClipParams& cp, const CellCtx& cc, Bounds& b,
                         int lane, bool& bad, uint32_t& st) {
    const int top = cp.pyr.nlev;  // virtual root level
    int sp = 0;
    if (lane == 0) P.stack[0] = (uint32_t)top << 27;
    sp = 1;
    __syncwarp();
    while (sp > 0) {
        uint32_t e = P.stack[sp - 1];
        sp--;
        __syncwarp();
        int l = (int)(e >> 27);
        int node = (int)(e & ((1u << 27) - 1));
        int cl = l - 1;
        int cdx = cp.pyr.dim[cl][0], cdy = cp.pyr.dim[cl][1], cdz = cp.pyr.dim[cl][2];
        int x0, y0, z0, nx, ny, nz;
        if (l == top) {
            x0 = y0 = z0 = 0;
            nx = cdx;
            ny = cdy;
            nz = cdz;
        } else {
            int pdx = cp.pyr.dim[l][0], pdy = cp.pyr.dim[l][1];
            int X = node % pdx, Y = (node / pdx) % pdy, Z = node / (pdx * pdy);
            x0 = 4 * X;
            y0 = 4 * Y;
            z0 = 4 * Z;
            nx = min(4, cdx - x0);
            ny = min(4, cdy - y0);
            nz = min(4, cdz - z0);
        }
        const int nch = nx * ny * nz;  // <= 64
        WCOUNT(P, 2, nch);
        WCOUNT(P, 7, 1);
        for (int base = 0; base < nch; base += 32) {
            int t = base + lane;
            bool surv = false;
            int cx = 0, cy = 0, cz = 0;
            if (t < nch) {
                cx = x0 + t % nx;
                cy = y0 + (t / nx) % ny;
                cz = z0 + t / (nx * ny);
                surv = !node_pruned(cp, b, cl, cx, cy, cz);
            }
            uint32_t sm = __ballot_sync(FULLMASK, surv);
            if (sm == 0) continue;
            if (cl > 0) {
                int n = __popc(sm);
                if (sp + n > STACK) {
                    st |= CS_CAPACITY | CS_CAP_STACK;
                    return false;
                }
                uint32_t below = (lane == 0) ? 0u : ((1u << lane) - 1u);
                if (surv)
                    P.stack[sp + __popc(sm & below)] =
                        ((uint32_t)cl << 27) | (uint32_t)(((int64_t)cz * cdy + cy) * cdx + cx);
                sp += n;
                __syncwarp();
                continue;
            }
            // surviving leaves: their seeds, one leaf per lane
            int64_t leaf = surv ? ((int64_t)cz * cp.G[1] + cy) * cp.G[0] + cx : -1;
            if (process_leaves<R, MODE>(P, cp, cc, b, leaf, lane, bad, st) == LEAF_STOP)
                return false;
        }
    }
    return true;
}

// Integrate the polytope and write the outputs of cell i; cen receives the centroid
// relative to the seed (units of a, every lane) and the return value says whether it
// is valid (positive finite volume).
template <typename R>
__device__ __noinline__ bool integrate(WarpPoly<R>& P, const ClipParams& cp, const Frame& fr,
                                       int64_t i, int lane, bool& bad, uint32_t& st,
                                       float* cen) {
    double vol6 = 0, mx = 0, my = 0, mz = 0, sx = 0, sy = 0, sz = 0, sabs = 0;
    constexpr int FPL = MAXP / 32;  // faces handled per lane
    // apex of the tetrahedron fans: the centre o of the vertices' bounding box, so the
    // determinants involve offsets of the cell's own size even when the cell lies far
    // from its seed (no cancellation of large terms in FP32)
    R o[3];
    {
        R mn[3] = {R(1e30), R(1e30), R(1e30)}, mx[3] = {R(-1e30), R(-1e30), R(-1e30)};
        for (int s2 = lane; s2 < P.nt; s2 += 32) {
            V3<R> v = P.v[s2];
            mn[0] = fmin(mn[0], v.x); mx[0] = fmax(mx[0], v.x);
            mn[1] = fmin(mn[1], v.y); mx[1] = fmax(mx[1], v.y);
            mn[2] = fmin(mn[2], v.z); mx[2] = fmax(mx[2], v.z);
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
            for (int q = 16; q > 0; q >>= 1) {
                mn[a] = fmin(mn[a], __shfl_xor_sync(FULLMASK, mn[a], q));
                mx[a] = fmax(mx[a], __shfl_xor_sync(FULLMASK, mx[a], q));
            }
            o[a] = R(0.5) * (mn[a] + mx[a]);
        }
    }
    int nf = 0;
    int32_t fj[FPL];
    double fc[FPL];
    const int nt = P.nt;
    for (int f = lane; f < ((P.np + 31) / 32) * 32; f += 32) {
        // faces f are handled in rounds so every lane runs the same triangle loop
        uint32_t ent[MAXFV];
        int m = 0;
        bool active = f < P.np;
        for (int s = 0; s < nt; s++) {
            uint32_t t = P.tri[s];
            if (!active) continue;
            uint32_t a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
            uint32_t x, y;
            if (a == (uint32_t)f) { x = b; y = c; }
            else if (b == (uint32_t)f) { x = c; y = a; }
            else if (c == (uint32_t)f) { x = a; y = b; }
            else continue;
            if (m < MAXFV) ent[m] = x | (y << 8) | ((uint32_t)s << 16);
            m++;
        }
        if (!active || m == 0) continue;
        if (m > MAXFV) {
            st |= CS_CAPACITY | CS_CAP_FACE;
            continue;
        }
        if (m < 3) {
            bad = true;
            continue;
        }
        // walk the cycle: the entry after (x, y) is the one whose x equals y
        int cur = 0;
        V3<R> v0 = P.v[ent[0] >> 16];
        v0.x -= o[0];
        v0.y -= o[1];
        v0.z -= o[2];
        V3<R> vp = v0;
        R Sx = 0, Sy = 0, Sz = 0;
        bool ok = true;
        for (int step = 1; step < m; step++) {
            uint32_t yv = (ent[cur] >> 8) & 0xff;
            int nxt = -1;
            for (int e2 = 0; e2 < m; e2++)
                if ((ent[e2] & 0xff) == yv) { nxt = e2; break; }
            if (nxt < 0 || nxt == 0) { ok = false; break; }
            cur = nxt;
            V3<R> vc = P.v[ent[cur] >> 16];
            vc.x -= o[0];
            vc.y -= o[1];
            vc.z -= o[2];
            if (step >= 2) {
                // fan triangle (v0, vp, vc) and tetrahedron (0, v0, vp, vc)
                R ax = vp.x - v0.x, ay = vp.y - v0.y, az = vp.z - v0.z;
                R bx = vc.x - v0.x, by = vc.y - v0.y, bz = vc.z - v0.z;
                R cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
                Sx += cx;
                Sy += cy;
                Sz += cz;
                // 6 |tet(o, v0, vp, vc)| = det(v0, vp, vc) with vertices relative to o
                double d6 = (double)(v0.x * cx + v0.y * cy + v0.z * cz);
                vol6 += d6;
                mx += d6 * ((double)v0.x + (double)vp.x + (double)vc.x);
                my += d6 * ((double)v0.y + (double)vp.y + (double)vc.y);
                mz += d6 * ((double)v0.z + (double)vp.z + (double)vc.z);
            }
            vp = vc;
        }
        if (ok && ((ent[cur] >> 8) & 0xff) != (ent[0] & 0xff)) ok = false;
        if (!ok) {
            bad = true;
            continue;
        }
        double ax2 = 0.5 * (double)Sx, ay2 = 0.5 * (double)Sy, az2 = 0.5 * (double)Sz;
        double A = sqrt(ax2 * ax2 + ay2 * ay2 + az2 * az2);
        sx += ax2;
        sy += ay2;
        sz += az2;
        sabs += A;
        int32_t j = P.pj[f];
        if (j >= 0 && A > 0.0) {
            if (nf < FPL) {
                fj[nf] = j;
                fc[nf] = A * cp.a / (double)P.plen[f];
            }
            nf++;
        }
    }
    vol6 = warp_sum(vol6);
    mx = warp_sum(mx);
    my = warp_sum(my);
    mz = warp_sum(mz);
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    sz = warp_sum(sz);
    sabs = warp_sum(sabs);
    // facets
    int incl = nf;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += y;
    }
    int total = __shfl_sync(FULLMASK, incl, 31);
    if (total > FCAP) st |= CS_CAPACITY | CS_CAP_FACE;
    else {
        int pos = incl - nf;
        for (int q = 0; q < nf && q < FPL; q++) {
            cp.fcol[i * FCAP + pos + q] = fj[q];
            cp.fval[i * FCAP + pos + q] = fc[q];
        }
    }
    double closure = sqrt(sx * sx + sy * sy + sz * sz);
    double tol = sizeof(R) == 4 ? 1e-4 : 1e-10;
    if (!(closure <= tol * sabs)) bad = true;
    double vol = vol6 / 6.0;
    if (!(vol > 0.0) || !isfinite(vol)) bad = true;
    // first moment about the seed = moment about o + (z + o) V (mx.. hold 24 x moment
    // about o; o is relative to the frame origin z)
    mx += 24.0 * (fr.zd[0] + (double)o[0]) * vol;
    my += 24.0 * (fr.zd[1] + (double)o[1]) * vol;
    mz += 24.0 * (fr.zd[2] + (double)o[2]) * vol;
    bad = __any_sync(FULLMASK, bad);
    uint32_t stall = __reduce_or_sync(FULLMASK, st);
    st = stall;
    const double mm[3] = {mx / 24.0, my / 24.0, mz / 24.0};
    const bool valid = vol > 0.0 && isfinite(vol);
    if (valid)
        for (int a = 0; a < 3; a++) cen[a] = (float)(mm[a] / vol);
    if (lane == 0) {
        double a3 = cp.a * cp.a * cp.a;
        double a4 = a3 * cp.a;
        cp.vol[i] = vol * a3;
        cp.m1[3 * i + 0] = mm[0] * a4;
        cp.m1[3 * i + 1] = mm[1] * a4;
        cp.m1[3 * i + 2] = mm[2] * a4;
        cp.fcnt[i] = total > FCAP ? FCAP : total;
        if (valid) {
            cp.anchor[3 * i + 0] = cen[0];
            cp.anchor[3 * i + 1] = cen[1];
            cp.anchor[3 * i + 2] = cen[2];
        }
    }
    return valid;
}

// the cell must stay inside the minimum-image range of every other seed: radius of
// the polytope about the seed (at -z in the polytope's frame) against half the box
template <typename R>
__device__ __forceinline__ bool cell_too_large(const WarpPoly<R>& P, const CellCtx& cc,
                                               float psimax_glob, float halfLmin, int lane) {
    V3<R> z0;
    z0.x = -(R)cc.fr.z[0];
    z0.y = -(R)cc.fr.z[1];
    z0.z = -(R)cc.fr.z[2];
    float R0 = (float)poly_radius(P, z0, lane);
    float dpsi = fmaxf(psimax_glob - cc.si.phi, 0.f);
    return R0 + sqrtf(R0 * R0 + 2.f * dpsi) > halfLmin * 0.9999f;
}

// An FP32 cell whose centroid lies more than this many spacings from its frame
// origin is clipped once more in a frame at the centroid (its rounding grows with the
// distance of its vertices from the origin)
constexpr float REFRAME_DIST = 0.5f;

// clip by a list of seeds (warp-uniform count): each lane builds one plane, then the
// warp clips by them in order
template <typename R>
__device__ __noinline__ int clip_list(WarpPoly<R>& P, const ClipParams& cp, const CellCtx& cc,
                                      const int32_t* list, int n, int lane, bool& bad) {
    for (int t0 = 0; t0 < n; t0 += 32) {
        int t = t0 + lane;
        V4<R> pl;
        pl.x = pl.y = pl.z = pl.w = R(0);
        R len = R(1);
        int32_t j = -1;
        if (t < n) {
            j = list[t];
            if (j >= 0 && j < cp.N && j != (int32_t)cc.i) build_plane(cp, cc, j, pl, len);
            else j = -1;  // out-of-range entry: a no-op plane far outside
        }
        int nk = min(32, n - t0);
        for (int u = 0; u < nk; u++) {
            V4<R> pn;
            pn.x = __shfl_sync(FULLMASK, pl.x, u);
            pn.y = __shfl_sync(FULLMASK, pl.y, u);
            pn.z = __shfl_sync(FULLMASK, pl.z, u);
            pn.w = __shfl_sync(FULLMASK, pl.w, u);
            R plen = __shfl_sync(FULLMASK, len, u);
            int32_t ju = __shfl_sync(FULLMASK, j, u);
            if (ju < 0) continue;
            // a seed already among the planes (the lists overlap) is not applied twice
            bool dup = false;
#pragma unroll
            for (int w = 0; w < MAXP / 32; w++)
                dup |= (lane + 32 * w < P.np && P.pj[lane + 32 * w] == ju);
            if (__any_sync(FULLMASK, dup)) continue;
            int rc = poly_clip_inl(P, pn, plen, ju, lane, bad);
            if (rc == CLIP_EMPTY || rc == CLIP_CAP) return rc;
        }
    }
    return CLIP_NONE;
}

// global upper bound of psi/a^2 (top pyramid level), every lane
__device__ __forceinline__ float top_psimax(const ClipParams& cp, int lane) {
    float m = -INFINITY;
    const int tl = cp.pyr.nlev - 1;
    const int ntop = cp.pyr.dim[tl][0] * cp.pyr.dim[tl][1] * cp.pyr.dim[tl][2];
    for (int t = lane; t < ntop; t += 32) m = fmaxf(m, cp.pyr.psimax[cp.pyr.off[tl] + t]);
    return warp_max(m);
}

// One work item w of a clipping pass: cell worklist[w] (or w), clipped by its first
// candidates, certified (pass 1) or walked (re-queue pass), integrated; outputs
// written, the cell queued for the next pass where needed.
template <typename R, int MODE>
__device__ __forceinline__ void process_cell(WarpPoly<R>& P, const ClipParams& cp, int64_t w,
                                             float psimax_glob, float halfLmin, int lane) {
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
    poly_init(P, cp, cc.fr.z, lane);
    // first candidates: the cell's facets in the previous diagram, then its k
    // nearest seeds
    int rc = CLIP_NONE;
#ifdef SDOT_DIAG_NO_PREV
    if (false) {
#else
    if (cp.facets_valid) {
#endif
        int nprev = min(cp.fcnt[i], FCAP);
        rc = clip_list(P, cp, cc, cp.fcol + i * FCAP, nprev, lane, bad);
    }
    // the k nearest seeds start every cell of the first diagram, and any cell with
    // no facets in the previous one
    const bool use_knn = !cp.facets_valid || cp.fcnt[i] == 0;
    if (use_knn && (rc == CLIP_NONE || rc == CLIP_CUT))
        rc = clip_list(P, cp, cc, cp.knn + i * cp.k, cp.k, lane, bad);
    if (rc == CLIP_EMPTY) st |= CS_EMPTY;
    if (rc == CLIP_CAP) st |= CS_CAPACITY | CS_CAP_POLY;
    if (!st) {
        Bounds b;
        for (int a = 0; a < 3; a++) {
            b.yabs[a] = (float)cc.si.c[a] * cp.ht[a] + cc.si.off[a];
            b.zf[a] = cc.fr.z[a];
        }
        b.psi_i = cc.si.phi;
        poly_bounds(P, cp, b, lane);
        bool done = true;
        if (MODE == MODE_FULL) done = ring_walk(P, cp, cc, b, zprev, lane, bad, st);
        if (done) done = traverse<R, MODE>(P, cp, cc, b, lane, bad, st);
#ifdef SDOT_COUNTERS
        __syncwarp();
        if (lane < 8) atomicAdd(&cp.counters64[lane], (unsigned long long)P.wc[lane]);
        __syncwarp();
        if (lane < 8) P.wc[lane] = 0;
        __syncwarp();
#endif
        if (!done && MODE == MODE_CERTIFY && (st & CS_UNCERTIFIED)) {
            if (lane == 0) {
                int32_t q = atomicAdd(cp.queue_cnt, 1);
                cp.queue_out[q] = (int32_t)i;
                cp.status[i] = (uint8_t)st;
            }
            return;
        }
    }
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
            __syncwarp();  // facets and counts written by integrate
            const int nf = min(cp.fcnt[i], FCAP);
            __syncwarp();
            cc.fr = make_frame(cp, cen);
            bad = false;
            st = 0;
            poly_init(P, cp, cc.fr.z, lane);
            int rc2 = clip_list(P, cp, cc, cp.fcol + i * FCAP, nf, lane, bad);
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
        cp.status[i] = (uint8_t)st;
        bool redo = sizeof(R) == 4 && (st & (CS_INCONSISTENT | CS_CAPACITY));
        if (redo) {
            int32_t q = atomicAdd(cp.q64_cnt, 1);
            cp.q64_out[q] = (int32_t)i;
        }
    }
}

template <typename R, int MODE>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, 4)
    clip_kernel(ClipParams cp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpPoly<R>* polys = reinterpret_cast<WarpPoly<R>*>(smem_raw);
    const int lane = threadIdx.x & 31;
    WarpPoly<R>& P = polys[threadIdx.x >> 5];
    const float psimax_glob = top_psimax(cp, lane);
    const float halfLmin = 0.5f * fminf(cp.Lt[0], fminf(cp.Lt[1], cp.Lt[2]));
    while (true) {
        int64_t w = 0;
        if (lane == 0) w = atomicAdd(cp.work_counter, 1);
        w = __shfl_sync(FULLMASK, w, 0);
        if (w >= cp.nwork) break;
        process_cell<R, MODE>(P, cp, w, psimax_glob, halfLmin, lane);
    }
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

template <typename R, int MODE>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, 4)
    clip_batch_kernel(ClipBatch bt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpPoly<R>* polys = reinterpret_cast<WarpPoly<R>*>(smem_raw);
    const int lane = threadIdx.x & 31;
    WarpPoly<R>& P = polys[threadIdx.x >> 5];
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
        const ClipParams cp = bt.jobs[lo];
        const float psimax_glob = top_psimax(cp, lane);
        const float halfLmin = 0.5f * fminf(cp.Lt[0], fminf(cp.Lt[1], cp.Lt[2]));
        process_cell<R, MODE>(P, cp, (int64_t)(w - bt.start[lo]), psimax_glob, halfLmin, lane);
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

int build_pyramid(DeviceState& d, const double* psi, cudaStream_t s) {
    const int64_t N = d.N;
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

template <typename R, int MODE>
static int launch_clip(const ClipParams& cp, cudaStream_t s) {
    const size_t smem = sizeof(WarpPoly<R>) * WARPS_PER_BLOCK;
    // kernel attributes and the persistent grid size, set once per instantiation
    // (thread-safe: contexts of different host threads launch concurrently)
    struct Setup {
        int blocks;
        cudaError_t err;
    };
    static const Setup setup = [smem] {
        Setup u{0, cudaSuccess};
        u.err = cudaFuncSetAttribute(clip_kernel<R, MODE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (u.err == cudaSuccess)
            u.err = cudaFuncSetAttribute(clip_kernel<R, MODE>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int per_sm = 0;
        if (u.err == cudaSuccess)
            u.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, clip_kernel<R, MODE>,
                                                                  WARPS_PER_BLOCK * 32, smem);
        if (per_sm < 1) per_sm = 1;
        u.blocks = per_sm * num_sms();
        return u;
    }();
    if (setup.err != cudaSuccess) {
        set_error(std::string("clip kernel setup: ") + cudaGetErrorString(setup.err));
        return SDOT_ERR_CUDA;
    }
    const int blocks = setup.blocks;
    int64_t need = (cp.nwork + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    int nb = (int)(need < blocks ? need : blocks);
    if (nb < 1) return SDOT_OK;
    clip_kernel<R, MODE><<<nb, WARPS_PER_BLOCK * 32, smem, s>>>(cp);
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
    cp.vol = d.vol;
    cp.m1 = d.m1;
    cp.anchor = d.anchor;
    cp.status = d.status;
    cp.fcnt = d.fcnt;
    cp.fcol = d.fcol;
    cp.fval = d.fval;
    cp.queue_out = d.queue;
    cp.queue_cnt = d.counters + 0;
    cp.q64_out = d.queue64;
    cp.q64_cnt = d.counters + 1;
    cp.counters64 = (unsigned long long*)(d.counters + 8);
    cp.work_counter = nullptr;
    cp.worklist = nullptr;
    cp.nwork = d.N;
    return cp;
}

int evaluate_cells(DeviceState& d, const double* psi, int precision, EvalResult* res,
                   cudaStream_t s) {
    int rc = build_pyramid(d, psi, s);
    if (rc) return rc;
    ClipParams cp = make_clip_params(d, psi);
    SDOT_CUDA_TRY(cudaMemsetAsync(d.counters, 0, 8 * sizeof(int32_t), s));

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
    rc = precision == SDOT_PREC_FP64 ? launch_clip<double, MODE_CERTIFY>(cp, s)
                                     : launch_clip<float, MODE_CERTIFY>(cp, s);
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
        rc = precision == SDOT_PREC_FP64 ? launch_clip<double, MODE_FULL>(cp, s)
                                         : launch_clip<float, MODE_FULL>(cp, s);
        if (rc) return rc;
        SDOT_CUDA_TRY(cudaMemcpyAsync(cnt, d.counters, 8, cudaMemcpyDeviceToHost, s));
        SDOT_CUDA_TRY(cudaStreamSynchronize(s));
    }
    cudaEventRecord(ep2, s);
    int64_t reclipped = cnt[1];
    // pass 3 (mixed): FP64 re-clip of cells failing the FP32 checks
    if (precision != SDOT_PREC_FP64 && reclipped > 0) {
        cp.work_counter = d.counters + 5;
        cp.worklist = d.queue64;
        cp.nwork = reclipped;
        rc = launch_clip<double, MODE_FULL>(cp, s);
        if (rc) return rc;
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
template <typename R, int MODE>
static int launch_clip_batch(const ClipBatch& bt, int64_t total, cudaStream_t s) {
    const size_t smem = sizeof(WarpPoly<R>) * WARPS_PER_BLOCK;
    struct Setup {
        int blocks;
        cudaError_t err;
    };
    static const Setup setup = [smem] {
        Setup u{0, cudaSuccess};
        u.err = cudaFuncSetAttribute(clip_batch_kernel<R, MODE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (u.err == cudaSuccess)
            u.err = cudaFuncSetAttribute(clip_batch_kernel<R, MODE>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int per_sm = 0;
        if (u.err == cudaSuccess)
            u.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, clip_batch_kernel<R, MODE>, WARPS_PER_BLOCK * 32, smem);
        if (per_sm < 1) per_sm = 1;
        u.blocks = per_sm * num_sms();
        return u;
    }();
    if (setup.err != cudaSuccess) {
        set_error(std::string("clip batch kernel setup: ") + cudaGetErrorString(setup.err));
        return SDOT_ERR_CUDA;
    }
    const int64_t need = (total + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    const int nb = (int)(need < setup.blocks ? need : setup.blocks);
    if (nb < 1) return SDOT_OK;
    clip_batch_kernel<R, MODE><<<nb, WARPS_PER_BLOCK * 32, smem, s>>>(bt);
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
template <typename R, int MODE>
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
    return launch_clip_batch<R, MODE>(bt, total, s);
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
        nwork[j] = ds[j]->N;
    }
    if ((rc = launch_table<float, MODE_CERTIFY>(cps, nwork, is32, 0, sc, s)) ||
        (rc = launch_table<double, MODE_CERTIFY>(cps, nwork, is64, 1, sc, s))) {
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
        nwork[j] = requeued[j];
        any = any || requeued[j] > 0;
    }
    // pass 2: the re-queued cells, full walk with clipping
    if (any) {
        if ((rc = launch_table<float, MODE_FULL>(cps, nwork, is32, 0, sc, s)) ||
            (rc = launch_table<double, MODE_FULL>(cps, nwork, is64, 1, sc, s))) {
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
        nwork[j] = is32[j] ? reclipped[j] : 0;
        any = any || nwork[j] > 0;
    }
    // pass 3: FP64 re-clip of the FP32 jobs' cells that failed the FP32 checks
    if (any && (rc = launch_table<double, MODE_FULL>(cps, nwork, all, 0, sc, s))) {
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
