/*
 * CPU oracle for semi-discrete optimal transport (Laguerre cells in a periodic box).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain FP64 statement of what
 * the CUDA path computes. Only the tests, the smoke check and the timed CPU
 * baseline of the benchmark may call it; the library never does. It shares no
 * code, header, table or helper with the CUDA sources.
 *
 * What it computes, with the passages of arXiv:2110.08868 it follows:
 *  - Laguerre (power) cell, eq. (laguerrecell):
 *        V_i = { q : 1/2|x_i - q|^2 - psi_i < 1/2|x_j - q|^2 - psi_j  for all j != i }.
 *    In local coordinates p = q - y_i and with d = (periodic image of y_j) - y_i this
 *    is the half-space p.d < 1/2|d|^2 + psi_i - psi_j. The cell is the intersection of
 *    these half-spaces over every j and every periodic image, i.e. the plain
 *    definition written out: each cell starts as the cube [-L/2, L/2]^3 (the bisectors
 *    with the seed's own six face images) and is clipped by one plane per candidate.
 *  - The integrals entering the semi-discrete dual, eq. (SDK): |V_i|,
 *    int_{V_i} p dp (first moment) and int_{V_i} 1/2 |p|^2 dp.
 *  - The facet areas A_ij, from which the second derivative of K is built
 *    (K is C^2, Sec. "Monge-Ampere-Kantorovich Reconstruction", smoothness paragraph).
 *  - Brute-force k nearest neighbours by minimum-image squared distance, ties
 *    broken by index.
 *
 * Two clipping modes give the same cell:
 *  - brute: every j != i and every one of the 27 image shifts of the
 *    minimum-image vector (plus the seed's own images), in increasing |d|;
 *    a plane is skipped only when its distance from the seed is >= the largest
 *    vertex radius R, in which case it provably cannot cut. Afterwards the cell
 *    is checked to be out of reach of every farther image.
 *  - certified: minimum-image candidates in increasing (|d|^2, j); stops when the
 *    next candidate distance D satisfies D >= R + sqrt(R^2 + 2 (psi_max - psi_i)),
 *    which bounds from below the distance of every unseen plane by R. Cells that
 *    cannot be certified inside the minimum-image range fall back to brute.
 *
 * Polyhedra are lists of convex faces (Sutherland-Hodgman on each face, the cap
 * polygon sorted by angle around the plane normal): a textbook representation.
 * Compile with -ffp-contract=off so the kNN distance is exactly
 * (dx*dx + dy*dy) + dz*dz in IEEE binary64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXF 400  /* faces per cell */
#define OR_MAXFV 96  /* vertices per face */
#define OR_MAXCAP 1024

enum { OR_OK = 0, OR_OVERFLOW = 1, OR_EMPTY = 2, OR_NOT_CERTIFIED = 4 };

typedef struct {
    int nf;
    int nv[OR_MAXF];
    int64_t tag[OR_MAXF];  /* -1: own image (box face); else neighbour index j */
    double dlen[OR_MAXF];  /* |d| of the plane's generating vector */
    double v[OR_MAXF][OR_MAXFV][3];
} poly_t;

/* minimum-image component: if dx > L/2 subtract L, else if dx < -L/2 add L */
static double wrap1(double dx, double L) {
    if (dx > 0.5 * L) return dx - L;
    if (dx < -0.5 * L) return dx + L;
    return dx;
}

static double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* The cube [-Lx/2,Lx/2] x ... with faces counter-clockwise seen from outside. */
static void poly_box(poly_t* P, const double* L) {
    double hx = 0.5 * L[0], hy = 0.5 * L[1], hz = 0.5 * L[2];
    double c[8][3];
    for (int k = 0; k < 8; k++) {
        c[k][0] = (k & 1) ? hx : -hx;
        c[k][1] = (k & 2) ? hy : -hy;
        c[k][2] = (k & 4) ? hz : -hz;
    }
    /* corner indices of each face, CCW about the outward normal */
    static const int F[6][4] = {
        {1, 3, 7, 5}, /* +x */
        {0, 4, 6, 2}, /* -x */
        {2, 6, 7, 3}, /* +y */
        {0, 1, 5, 4}, /* -y */
        {4, 5, 7, 6}, /* +z */
        {0, 2, 3, 1}, /* -z */
    };
    P->nf = 6;
    for (int f = 0; f < 6; f++) {
        P->nv[f] = 4;
        P->tag[f] = -1;
        P->dlen[f] = L[f / 2];
        for (int k = 0; k < 4; k++) memcpy(P->v[f][k], c[F[f][k]], sizeof(double) * 3);
    }
}

typedef struct { double ang; double p[3]; } capv_t;

static int cmp_cap(const void* a, const void* b) {
    double x = ((const capv_t*)a)->ang, y = ((const capv_t*)b)->ang;
    return (x > y) - (x < y);
}

/*
 * Clip P by the half-space p.n <= b (n not normalised). Returns 0 if nothing was
 * cut, 1 if cut, -1 on capacity overflow. Q is scratch of the same type; on return P holds
 * the result.
 */
static int poly_clip(poly_t* P, poly_t* Q, const double* n, double b, int64_t tag,
                     double dlen, capv_t* cap) {
    int any_out = 0;
    for (int f = 0; f < P->nf && !any_out; f++)
        for (int k = 0; k < P->nv[f]; k++)
            if (dot3(P->v[f][k], n) - b > 0.0) { any_out = 1; break; }
    if (!any_out) return 0;

    int ncap = 0;
    Q->nf = 0;
    for (int f = 0; f < P->nf; f++) {
        int m = P->nv[f];
        int g = Q->nf;
        int cnt = 0;
        if (g >= OR_MAXF) return -1;
        for (int k = 0; k < m; k++) {
            const double* A = P->v[f][k];
            const double* B = P->v[f][(k + 1) % m];
            double sa = dot3(A, n) - b;
            double sb = dot3(B, n) - b;
            int ina = sa <= 0.0, inb = sb <= 0.0;
            if (ina) {
                if (cnt >= OR_MAXFV) return -1;
                memcpy(Q->v[g][cnt++], A, sizeof(double) * 3);
            }
            if (ina != inb) {
                /* intersection, always computed from the inside end point so that
                   the two faces sharing this edge produce bit-identical points */
                const double* I = ina ? A : B;
                const double* O = ina ? B : A;
                double si = ina ? sa : sb, so = ina ? sb : sa;
                double t = si / (si - so);
                double p[3];
                for (int c = 0; c < 3; c++) p[c] = I[c] + t * (O[c] - I[c]);
                if (cnt >= OR_MAXFV) return -1;
                if (cnt == 0 || memcmp(Q->v[g][cnt - 1], p, sizeof p) != 0)
                    memcpy(Q->v[g][cnt++], p, sizeof p);
                int dup = 0;
                for (int c = 0; c < ncap; c++)
                    if (memcmp(cap[c].p, p, sizeof p) == 0) { dup = 1; break; }
                if (!dup) {
                    if (ncap >= OR_MAXCAP) return -1;
                    memcpy(cap[ncap++].p, p, sizeof p);
                }
            }
        }
        /* drop a closing duplicate */
        if (cnt > 1 && memcmp(Q->v[g][cnt - 1], Q->v[g][0], sizeof(double) * 3) == 0) cnt--;
        if (cnt >= 3) {
            if (Q->nf >= OR_MAXF) return -1;
            Q->nv[g] = cnt;
            Q->tag[g] = P->tag[f];
            Q->dlen[g] = P->dlen[f];
            Q->nf++;
        }
    }
    if (ncap >= 3) {
        /* cap polygon: sort by angle about n, counter-clockwise seen from +n */
        double nn = sqrt(dot3(n, n));
        double nh[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
        double ctr[3] = {0, 0, 0};
        for (int c = 0; c < ncap; c++)
            for (int e = 0; e < 3; e++) ctr[e] += cap[c].p[e];
        for (int e = 0; e < 3; e++) ctr[e] /= ncap;
        double t0[3] = {1, 0, 0};
        if (fabs(nh[0]) > 0.6) { t0[0] = 0; t0[1] = 1; }
        double u[3], w[3];
        cross3(nh, t0, u);
        double un = sqrt(dot3(u, u));
        for (int e = 0; e < 3; e++) u[e] /= un;
        cross3(nh, u, w);
        for (int c = 0; c < ncap; c++) {
            double r[3] = {cap[c].p[0] - ctr[0], cap[c].p[1] - ctr[1], cap[c].p[2] - ctr[2]};
            cap[c].ang = atan2(dot3(r, w), dot3(r, u));
        }
        qsort(cap, ncap, sizeof(capv_t), cmp_cap);
        if (Q->nf >= OR_MAXF || ncap > OR_MAXFV) return -1;
        int g = Q->nf++;
        Q->nv[g] = ncap;
        Q->tag[g] = tag;
        Q->dlen[g] = dlen;
        for (int c = 0; c < ncap; c++) memcpy(Q->v[g][c], cap[c].p, sizeof(double) * 3);
    }
    /* P <- Q */
    P->nf = Q->nf;
    for (int f = 0; f < Q->nf; f++) {
        P->nv[f] = Q->nv[f];
        P->tag[f] = Q->tag[f];
        P->dlen[f] = Q->dlen[f];
        memcpy(P->v[f], Q->v[f], sizeof(double) * 3 * Q->nv[f]);
    }
    return 1;
}

static double poly_radius(const poly_t* P) {
    double r2 = 0.0;
    for (int f = 0; f < P->nf; f++)
        for (int k = 0; k < P->nv[f]; k++) {
            double s = dot3(P->v[f][k], P->v[f][k]);
            if (s > r2) r2 = s;
        }
    return sqrt(r2);
}

typedef struct {
    double d2;
    int64_t j;
    double d[3];
} cand_t;

static int cmp_cand(const void* a, const void* b) {
    const cand_t* x = (const cand_t*)a;
    const cand_t* y = (const cand_t*)b;
    if (x->d2 < y->d2) return -1;
    if (x->d2 > y->d2) return 1;
    return (x->j > y->j) - (x->j < y->j);
}

/*
 * Integrals over the polytope (local coordinates, seed at the origin), by a fan of
 * tetrahedra (origin, v0, vk, vk+1) over each face:
 *   |T| = det(v0, vk, vk+1)/6, int_T p = |T| (v0+vk+vk+1)/4,
 *   int_T |p|^2 = |T|/20 (|v0|^2+|vk|^2+|vk+1|^2 + |v0+vk+vk+1|^2).
 * Signed volumes keep this exact when the seed lies outside its own cell.
 */
static void poly_integrals(const poly_t* P, double* vol, double* m1, double* i2) {
    double V = 0, M[3] = {0, 0, 0}, I = 0;
    for (int f = 0; f < P->nf; f++) {
        const double* a = P->v[f][0];
        for (int k = 1; k + 1 < P->nv[f]; k++) {
            const double* b = P->v[f][k];
            const double* c = P->v[f][k + 1];
            double bc[3];
            cross3(b, c, bc);
            double t = dot3(a, bc) / 6.0;
            double s[3] = {a[0] + b[0] + c[0], a[1] + b[1] + c[1], a[2] + b[2] + c[2]};
            V += t;
            for (int e = 0; e < 3; e++) M[e] += t * s[e] / 4.0;
            I += t / 20.0 * (dot3(a, a) + dot3(b, b) + dot3(c, c) + dot3(s, s));
        }
    }
    *vol = V;
    for (int e = 0; e < 3; e++) m1[e] = M[e];
    *i2 = I;
}

/* area of a planar polygon: half the norm of sum v_k x v_{k+1} */
static double face_area(const poly_t* P, int f) {
    double A[3] = {0, 0, 0};
    int m = P->nv[f];
    for (int k = 0; k < m; k++) {
        double c[3];
        cross3(P->v[f][k], P->v[f][(k + 1) % m], c);
        for (int e = 0; e < 3; e++) A[e] += c[e];
    }
    return 0.5 * sqrt(dot3(A, A));
}

/* clip P by the plane of candidate (d, j); skip planes at distance >= R.
   Returns OR_OK or OR_OVERFLOW. */
static int clip_cand(poly_t* P, poly_t* Q, capv_t* cap, const double* d, int64_t j,
                     double psi_i, double psi_j, double* R) {
    double d2 = dot3(d, d);
    double dl = sqrt(d2);
    double b = 0.5 * d2 + psi_i - psi_j;
    if (b >= *R * dl) return 0; /* h = b/|d| >= R: no vertex is beyond the plane */
    int r = poly_clip(P, Q, d, b, j, dl, cap);
    if (r == 1) *R = poly_radius(P);
    return r < 0 ? OR_OVERFLOW : OR_OK;
}

typedef struct {
    poly_t P, Q;
    capv_t cap[OR_MAXCAP];
    cand_t* cand;
    int64_t ncand_cap;
} work_t;

static int cell_brute(work_t* W, int64_t i, int64_t N, const double* pos, const double* psi,
                      const double* L, double dpsi_max) {
    const double* yi = pos + 3 * i;
    double Lmin = fmin(L[0], fmin(L[1], L[2]));
    poly_box(&W->P, L);
    double R = poly_radius(&W->P);
    /* shells of image shifts: shell s holds the shifts with max|shift| == s; every
       image outside shells 0..s lies at |d| >= (s + 1/2) min(L) */
    for (int sh = 1; sh <= 4; sh++) {
        int64_t nc = 0;
        int w = 2 * sh + 1;
        for (int64_t j = 0; j < N; j++) {
            double m[3];
            for (int e = 0; e < 3; e++) m[e] = wrap1(pos[3 * j + e] - yi[e], L[e]);
            for (int s = 0; s < w * w * w; s++) {
                int sx = s % w - sh, sy = (s / w) % w - sh, sz = s / (w * w) - sh;
                int cheb = abs(sx) > abs(sy) ? abs(sx) : abs(sy);
                if (abs(sz) > cheb) cheb = abs(sz);
                if (sh == 1 ? cheb > 1 : cheb != sh) continue;
                if (j == i && cheb == 0) continue;
                if (nc >= W->ncand_cap) return OR_OVERFLOW;
                cand_t* c = &W->cand[nc++];
                c->d[0] = m[0] + sx * L[0];
                c->d[1] = m[1] + sy * L[1];
                c->d[2] = m[2] + sz * L[2];
                c->d2 = dot3(c->d, c->d);
                c->j = j;
            }
        }
        qsort(W->cand, nc, sizeof(cand_t), cmp_cand);
        for (int64_t c = 0; c < nc; c++) {
            const cand_t* k = &W->cand[c];
            /* own images have a zero psi difference; the six face images are the
               box faces already, the others are clipped like any plane */
            int64_t tag = (k->j == i) ? -1 : k->j;
            double pj = (k->j == i) ? psi[i] : psi[k->j];
            if (clip_cand(&W->P, &W->Q, W->cap, k->d, tag, psi[i], pj, &R) == OR_OVERFLOW)
                return OR_OVERFLOW;
            if (W->P.nf == 0) return OR_EMPTY;
        }
        if (R + sqrt(R * R + 2.0 * dpsi_max) <= (sh + 0.5) * Lmin) return OR_OK;
    }
    return OR_NOT_CERTIFIED;
}

static int cell_certified(work_t* W, int64_t i, int64_t N, const double* pos,
                          const double* psi, const double* L, double dpsi_max) {
    int64_t nc = 0;
    const double* yi = pos + 3 * i;
    for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        cand_t* c = &W->cand[nc++];
        for (int e = 0; e < 3; e++) c->d[e] = wrap1(pos[3 * j + e] - yi[e], L[e]);
        c->d2 = (c->d[0] * c->d[0] + c->d[1] * c->d[1]) + c->d[2] * c->d[2];
        c->j = j;
    }
    qsort(W->cand, nc, sizeof(cand_t), cmp_cand);
    poly_box(&W->P, L);
    double R = poly_radius(&W->P);
    /* every non-minimum image has one component of magnitude >= L/2 */
    double Dimg = 0.5 * fmin(L[0], fmin(L[1], L[2]));
    for (int64_t c = 0; c <= nc; c++) {
        double D = (c < nc) ? sqrt(W->cand[c].d2) : INFINITY;
        if (D > Dimg) D = Dimg;
        if (D >= R + sqrt(R * R + 2.0 * dpsi_max)) return OR_OK;
        if (c == nc) break;
        const cand_t* k = &W->cand[c];
        if (clip_cand(&W->P, &W->Q, W->cap, k->d, k->j, psi[i], psi[k->j], &R) == OR_OVERFLOW)
            return OR_OVERFLOW;
        if (W->P.nf == 0) return OR_EMPTY;
    }
    return OR_NOT_CERTIFIED;
}

/*
 * One cell. Outputs: vol, m1[3] (int p dp), i2 (int 1/2|p|^2 dp), radius, and
 * up to fmax facets (j, area, |d|) with non-negative tag. Returns status.
 */
static int one_cell(work_t* W, int64_t i, int64_t N, const double* pos, const double* psi,
                    const double* L, double psi_max, int mode, double* vol, double* m1,
                    double* i2, double* radius, int fmax, int64_t* fj, double* farea,
                    double* fdist, int* nfac) {
    double dpsi = psi_max - psi[i];
    if (dpsi < 0) dpsi = 0;
    int st;
    if (mode == 1) st = cell_certified(W, i, N, pos, psi, L, dpsi);
    if (mode != 1 || st == OR_NOT_CERTIFIED) {
        /* brute force is only meant for small N (the largest image shell holds
           9^3 - 7^3 = 386 shifts per seed) */
        if (N > 200000) return OR_NOT_CERTIFIED;
        if (W->ncand_cap < 386 * N) {
            free(W->cand);
            W->ncand_cap = 386 * N;
            W->cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)W->ncand_cap);
        }
        st = cell_brute(W, i, N, pos, psi, L, dpsi);
    }
    if (st == OR_EMPTY) {
        *vol = 0; m1[0] = m1[1] = m1[2] = 0; *i2 = 0; *radius = 0; *nfac = 0;
        return st;
    }
    if (st == OR_OVERFLOW) return st;
    double v, i2h;
    poly_integrals(&W->P, &v, m1, &i2h);
    *vol = v;
    *i2 = 0.5 * i2h;
    *radius = poly_radius(&W->P);
    int nf = 0;
    for (int f = 0; f < W->P.nf; f++) {
        if (W->P.tag[f] < 0) continue;
        if (nf >= fmax) return OR_OVERFLOW;
        fj[nf] = W->P.tag[f];
        farea[nf] = face_area(&W->P, f);
        fdist[nf] = W->P.dlen[f];
        nf++;
    }
    *nfac = nf;
    return st;
}

/*
 * Laguerre cells for the listed seeds (or all if idx == NULL).
 * mode 0 = brute, 1 = certified. Facet arrays are [n_out * fmax].
 * status[n_out] receives per-cell status. Returns the OR of all statuses.
 */
int oracle_cells(int64_t N, const double* pos, const double* psi, const double* L,
                 int mode, int64_t n_out, const int64_t* idx, double* vol, double* m1,
                 double* i2, double* radius, int fmax, int64_t* fj, double* farea,
                 double* fdist, int* nfac, int* status) {
    double psi_max = -INFINITY;
    for (int64_t j = 0; j < N; j++)
        if (psi[j] > psi_max) psi_max = psi[j];
    int agg = 0;
    int64_t cand_cap = (mode == 1 ? N : 386 * N);
#pragma omp parallel reduction(| : agg)
    {
        work_t* W = (work_t*)malloc(sizeof(work_t));
        W->cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)cand_cap);
        W->ncand_cap = cand_cap;
#pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < n_out; t++) {
            int64_t i = idx ? idx[t] : t;
            int st = one_cell(W, i, N, pos, psi, L, psi_max, mode, vol + t, m1 + 3 * t,
                              i2 + t, radius + t, fmax, fj + (size_t)t * fmax,
                              farea + (size_t)t * fmax, fdist + (size_t)t * fmax,
                              nfac + t);
            status[t] = st;
            agg |= st;
        }
        free(W->cand);
        free(W);
    }
    return agg;
}

/*
 * Brute-force k nearest neighbours for the listed queries (all if idx == NULL):
 * all j != i sorted by (d2, j) with d2 = (dx*dx + dy*dy) + dz*dz of the
 * minimum-image difference y_j - y_i. out[n_out * k] (int64), d2out may be NULL.
 */
int oracle_knn(int64_t N, const double* pos, const double* L, int k, int64_t n_out,
               const int64_t* idx, int64_t* out, double* d2out) {
    if (k > N - 1) return -1;
#pragma omp parallel
    {
        cand_t* c = (cand_t*)malloc(sizeof(cand_t) * (size_t)N);
#pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < n_out; t++) {
            int64_t i = idx ? idx[t] : t;
            int64_t nc = 0;
            for (int64_t j = 0; j < N; j++) {
                if (j == i) continue;
                double dx = wrap1(pos[3 * j + 0] - pos[3 * i + 0], L[0]);
                double dy = wrap1(pos[3 * j + 1] - pos[3 * i + 1], L[1]);
                double dz = wrap1(pos[3 * j + 2] - pos[3 * i + 2], L[2]);
                c[nc].d2 = (dx * dx + dy * dy) + dz * dz;
                c[nc].j = j;
                nc++;
            }
            qsort(c, nc, sizeof(cand_t), cmp_cand);
            for (int q = 0; q < k; q++) {
                out[(size_t)t * k + q] = c[q].j;
                if (d2out) d2out[(size_t)t * k + q] = c[q].d2;
            }
        }
        free(c);
    }
    return 0;
}

/*
 * Kantorovich potential at tau_I on a mesh (Sec. "Monge-Ampere-Kantorovich
 * Reconstruction", the Legendre transform of psi):
 *     phi_I(q) = min_i [1/2 |q - x_i|^2 - psi_i]  (minimum image),
 * attained in the Laguerre cell i(q) that contains q. Evaluated by brute force over all
 * seeds at the M^3 mesh points q = (m + 1/2) L / M; owner[m] = i(q), the lowest index on
 * a tie.
 */
int oracle_potential_mesh(int64_t N, const double* pos, const double* psi, const double* L,
                          int M, double* phi, int64_t* owner) {
    if (M < 1) return -1;
    const int64_t nm = (int64_t)M * M * M;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < nm; m++) {
        const int64_t mx = m % M, my = (m / M) % M, mz = m / ((int64_t)M * M);
        const double q[3] = {(mx + 0.5) * L[0] / M, (my + 0.5) * L[1] / M, (mz + 0.5) * L[2] / M};
        double best = INFINITY;
        int64_t arg = -1;
        for (int64_t j = 0; j < N; j++) {
            double s = 0.0;
            for (int e = 0; e < 3; e++) {
                const double d = wrap1(q[e] - pos[3 * j + e], L[e]);
                s += d * d;
            }
            const double f = 0.5 * s - psi[j];
            if (f < best) {
                best = f;
                arg = j;
            }
        }
        phi[m] = best;
        owner[m] = arg;
    }
    return 0;
}

/*
 * Zel'dovich move of the cells and their mass density on an Eulerian mesh (Sec.
 * "Monge-Ampere-Kantorovich Reconstruction", last paragraph; Fig. 1). The point q of
 * cell V_i moves to q + lambda (x_i - q) (lambda = D(tau)/D(tau_F), 0 <= lambda < 1),
 * so the cell becomes its image under the homothety of ratio 1 - lambda centred at
 * x_i and carries the mass m_i spread uniformly over it. The mass of mesh voxel v is
 *     sum_i m_i |h_i(V_i) cap v| / |h_i(V_i)| = sum_i m_i |V_i cap h_i^-1(v)| / |V_i|,
 * computed here by clipping each cell with the six planes of h_i^-1(v) for every voxel
 * its moved bounding box meets. rho[v] = mass / voxel volume (M^3 voxels of side L/M).
 * Cells are the certified cells of oracle_cells; the sums run serially over cells in
 * index order.
 */
int oracle_deposit(int64_t N, const double* pos, const double* psi, const double* mass,
                   const double* L, int M, double lambda, double* rho) {
    if (M < 1 || !(lambda >= 0.0 && lambda < 1.0)) return -1;
    const int64_t nm = (int64_t)M * M * M;
    for (int64_t m = 0; m < nm; m++) rho[m] = 0.0;
    double psi_max = -INFINITY;
    for (int64_t j = 0; j < N; j++)
        if (psi[j] > psi_max) psi_max = psi[j];
    work_t* W = (work_t*)malloc(sizeof(work_t));
    poly_t* R = (poly_t*)malloc(sizeof(poly_t));
    W->cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)N);
    W->ncand_cap = N;
    int agg = 0;
    const double s = 1.0 - lambda;
    const double h[3] = {L[0] / M, L[1] / M, L[2] / M};
    for (int64_t i = 0; i < N && !(agg & OR_OVERFLOW); i++) {
        double dpsi = psi_max - psi[i];
        if (dpsi < 0) dpsi = 0;
        int st = cell_certified(W, i, N, pos, psi, L, dpsi);
        if (st == OR_NOT_CERTIFIED) {
            if (W->ncand_cap < 386 * N) {
                free(W->cand);
                W->ncand_cap = 386 * N;
                W->cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)W->ncand_cap);
            }
            st = cell_brute(W, i, N, pos, psi, L, dpsi);
        }
        agg |= st;
        if (st != OR_OK) continue;
        double vol, m1[3], i2;
        poly_integrals(&W->P, &vol, m1, &i2);
        if (!(vol > 0.0)) continue;
        /* local bounding box (p = q - x_i), its moved image, the voxels it meets */
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int f = 0; f < W->P.nf; f++)
            for (int k = 0; k < W->P.nv[f]; k++)
                for (int e = 0; e < 3; e++) {
                    lo[e] = fmin(lo[e], W->P.v[f][k][e]);
                    hi[e] = fmax(hi[e], W->P.v[f][k][e]);
                }
        const double* y = pos + 3 * i;
        int64_t v0[3], v1[3];
        for (int e = 0; e < 3; e++) {
            v0[e] = (int64_t)floor((y[e] + s * lo[e]) / h[e]);
            v1[e] = (int64_t)floor((y[e] + s * hi[e]) / h[e]);
        }
        for (int64_t vz = v0[2]; vz <= v1[2]; vz++)
            for (int64_t vy = v0[1]; vy <= v1[1]; vy++)
                for (int64_t vx = v0[0]; vx <= v1[0]; vx++) {
                    const int64_t vv[3] = {vx, vy, vz};
                    /* copy the cell, clip it by the voxel pulled back by the homothety */
                    R->nf = W->P.nf;
                    for (int f = 0; f < W->P.nf; f++) {
                        R->nv[f] = W->P.nv[f];
                        R->tag[f] = W->P.tag[f];
                        R->dlen[f] = W->P.dlen[f];
                        memcpy(R->v[f], W->P.v[f], sizeof(double) * 3 * W->P.nv[f]);
                    }
                    int empty = 0;
                    for (int e = 0; e < 3 && !empty; e++) {
                        const double blo = (vv[e] * h[e] - y[e]) / s;
                        const double bhi = ((vv[e] + 1) * h[e] - y[e]) / s;
                        double n[3] = {0, 0, 0};
                        n[e] = 1.0;
                        if (poly_clip(R, &W->Q, n, bhi, -2, 1.0, W->cap) < 0) agg |= OR_OVERFLOW;
                        n[e] = -1.0;
                        if (R->nf > 0 && poly_clip(R, &W->Q, n, -blo, -2, 1.0, W->cap) < 0)
                            agg |= OR_OVERFLOW;
                        if (R->nf == 0) empty = 1;
                    }
                    if (empty) continue;
                    double v2, mm[3], ii;
                    poly_integrals(R, &v2, mm, &ii);
                    if (!(v2 > 0.0)) continue;
                    const int64_t wx = ((vx % M) + M) % M, wy = ((vy % M) + M) % M,
                                  wz = ((vz % M) + M) % M;
                    rho[(wz * M + wy) * M + wx] += mass[i] * (v2 / vol);
                }
    }
    free(W->cand);
    free(W);
    free(R);
    const double vox = h[0] * h[1] * h[2];
    for (int64_t m = 0; m < nm; m++) rho[m] /= vox;
    return agg & OR_OVERFLOW ? -2 : 0;
}
