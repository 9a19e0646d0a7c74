"""CPU oracle for semi-discrete optimal transport — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. The library never does, and nothing here
imports the library: the geometry lives in ``oracle.c`` (plain C, FP64) and the
linear algebra below is numpy/scipy.

Passages of arXiv:2110.08868 followed:
  * eq. (SDK): K(psi) = sum_i int_{V_i} [1/2|x_i - q|^2 - psi_i] dq + sum_i m_i psi_i
  * eq. (laguerrecell): the Laguerre cells V_i^psi
  * Sec. "Monge-Ampere-Kantorovich Reconstruction", concavity/smoothness paragraph:
    K is concave and C^2, so it is maximised by a Newton method using first and
    second derivatives; the paragraph before it: maximise K with no empty cell
  * last paragraph of the same section: each cell V_i is mapped to x_i, so the
    Zel'dovich displacement of the mass element is x_i - (centroid of V_i).

Derivatives used (derived from eq. SDK and eq. laguerrecell, not printed in the
paper): dK/dpsi_i = m_i - |V_i|; for j != i, d|V_i|/dpsi_j = -A_ij/|d_ij| where
A_ij is the area of the facet shared with (an image of) j and d_ij the vector
between the two seeds; so the Hessian of K is -L with L the weighted graph
Laplacian L_ij = -A_ij/|d_ij|, L_ii = sum_j A_ij/|d_ij|.

Damped Newton reading (the paper only cites Kitagawa-Merigot-Thibert): eps0 =
1/2 min(min_i |V_i(psi0)|, min_i m_i); the step alpha = 1, 1/2, 1/4, ... is the
first for which min_i |V_i| >= eps0 and ||m - V||_2 <= (1 - alpha/2)||m - V(psi)||_2.
Stop when max_i |m_i - V_i| / m_i <= tol. The gauge sum(psi) = 0 is fixed after
every step (K is invariant under psi -> psi + c).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

FMAX = 384  # facets kept per cell

ST_OVERFLOW, ST_EMPTY, ST_NOT_CERTIFIED = 1, 2, 4


def build(force=False):
    """Compile oracle.c into liboracle.so beside it (gcc, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_cells.argtypes = [i64, P, P, P, ctypes.c_int, i64, P, P, P, P, P,
                                     ctypes.c_int, P, P, P, P, P]
        lib.oracle_cells.restype = ctypes.c_int
        lib.oracle_knn.argtypes = [i64, P, P, ctypes.c_int, i64, P, P, P]
        lib.oracle_knn.restype = ctypes.c_int
        lib.oracle_potential_mesh.argtypes = [i64, P, P, P, ctypes.c_int, P, P]
        lib.oracle_potential_mesh.restype = ctypes.c_int
        lib.oracle_deposit.argtypes = [i64, P, P, P, P, ctypes.c_int, ctypes.c_double, P]
        lib.oracle_deposit.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _box(box):
    b = np.asarray(box, dtype=np.float64).reshape(-1)
    if b.size == 1:
        b = np.repeat(b, 3)
    return np.ascontiguousarray(b)


def knn(pos, box, k, idx=None):
    """k nearest neighbours of each query by (minimum-image d^2, index).

    Returns (nbr[n_out, k] int64, d2[n_out, k] float64).
    """
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    N = pos.shape[0]
    L = _box(box)
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
    n_out = N if idx is None else idx.size
    out = np.empty((n_out, k), dtype=np.int64)
    d2 = np.empty((n_out, k), dtype=np.float64)
    rc = lib.oracle_knn(N, _ptr(pos), _ptr(L), k, n_out, _ptr(idx), _ptr(out), _ptr(d2))
    if rc != 0:
        raise ValueError("k must be < N")
    return out, d2


def cells(pos, psi, box, mode="certified", idx=None):
    """Laguerre cells of eq. (laguerrecell) for the queried seeds (all by default).

    Returns a dict with, per queried cell t (seed i = idx[t]):
      vol[t] = |V_i|, m1[t] = int_{V_i} (q - y_i) dq, i2[t] = int 1/2|q - y_i|^2 dq,
      radius[t] = max vertex distance from y_i, and facet lists (fj, farea, fdist, nfac)
      where fj are neighbour indices, farea the facet areas A_ij and fdist |d_ij|.
    """
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    N = pos.shape[0]
    L = _box(box)
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
    n_out = N if idx is None else idx.size
    vol = np.zeros(n_out)
    m1 = np.zeros((n_out, 3))
    i2 = np.zeros(n_out)
    rad = np.zeros(n_out)
    fj = np.full((n_out, FMAX), -1, dtype=np.int64)
    fa = np.zeros((n_out, FMAX))
    fd = np.zeros((n_out, FMAX))
    nf = np.zeros(n_out, dtype=np.int32)
    st = np.zeros(n_out, dtype=np.int32)
    m = {"brute": 0, "certified": 1}[mode]
    lib.oracle_cells(N, _ptr(pos), _ptr(psi), _ptr(L), m, n_out, _ptr(idx), _ptr(vol),
                     _ptr(m1), _ptr(i2), _ptr(rad), FMAX, _ptr(fj), _ptr(fa), _ptr(fd),
                     _ptr(nf), _ptr(st))
    if np.any(st & ST_OVERFLOW):
        raise RuntimeError("oracle polytope capacity exceeded")
    if np.any(st & ST_NOT_CERTIFIED):
        raise RuntimeError("oracle cell not certified within the 27 periodic images")
    return dict(vol=vol, m1=m1, i2=i2, radius=rad, fj=fj, farea=fa, fdist=fd, nfac=nf,
                status=st)


def hessian_laplacian(c, N):
    """Assemble L (= -Hessian of K) as scipy CSR from the facet lists of all cells.

    L_ij = -sum over facets of cell i with neighbour j of A/|d|; L_ii = -sum_j L_ij.
    Facets of zero area are dropped.
    """
    rows, cols, vals = [], [], []
    for i in range(N):
        n = c["nfac"][i]
        for f in range(n):
            a = c["farea"][i, f]
            if a <= 0.0:
                continue
            rows.append(i)
            cols.append(int(c["fj"][i, f]))
            vals.append(-a / c["fdist"][i, f])
    off = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    off.sum_duplicates()
    diag = -np.asarray(off.sum(axis=1)).ravel()
    return (off + sp.diags(diag)).tocsr()


def laguerre(pos, psi, box, nu=None, mode="certified", with_hessian=True):
    """Everything one Newton step needs at psi.

    Returns dict: vol, centroid (absolute, wrapped into the box), K (eq. SDK; needs
    nu), grad = nu - vol, L (scipy CSR, if with_hessian), and the raw cell dict.
    """
    pos = np.asarray(pos, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    N = pos.shape[0]
    L = _box(box)
    c = cells(pos, psi, L, mode)
    vol = c["vol"]
    with np.errstate(invalid="ignore", divide="ignore"):
        loc = c["m1"] / vol[:, None]
    cen = np.mod(pos + loc, L)
    cen[cen >= L] -= np.broadcast_to(L, cen.shape)[cen >= L]
    out = dict(vol=vol, centroid=cen, local_centroid=loc, cells=c)
    if nu is not None:
        nu = np.asarray(nu, dtype=np.float64)
        # eq. (SDK): sum_i int_{V_i} [1/2|x_i - q|^2 - psi_i] dq + sum_i m_i psi_i
        out["K"] = float(np.sum(c["i2"] - psi * vol) + np.sum(nu * psi))
        out["grad"] = nu - vol
    if with_hessian:
        out["L"] = hessian_laplacian(c, N)
    return out


def _newton_direction(Lm, g):
    """Solve L delta = g on the consistent singular system (mean-zero rhs).

    One unknown is pinned to zero (delta_0 = 0) and the rest solved directly;
    the result is then shifted to mean zero. Direct sparse LU: exact up to rounding.
    """
    N = g.size
    g = g - g.mean()
    A = Lm[1:, 1:].tocsc()
    d = np.zeros(N)
    d[1:] = spla.spsolve(A, g[1:])
    return d - d.mean()


def solve(pos, nu, box, tol=1e-4, psi0=None, mode="certified", maxit=100, verbose=False):
    """Damped Newton maximisation of K (eq. SDK) until max|m - V|/m <= tol.

    Returns (psi, info) with info holding vol, centroid, displacement, iterations,
    line-search evaluations and the error history.
    """
    pos = np.asarray(pos, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    N = pos.shape[0]
    psi = np.zeros(N) if psi0 is None else np.array(psi0, dtype=np.float64)
    psi -= psi.mean()
    ev = laguerre(pos, psi, box, nu, mode)
    eps0 = 0.5 * min(ev["vol"].min(), nu.min())
    hist = []
    n_eval = 1
    it = 0
    while True:
        g = ev["grad"]
        err = float(np.max(np.abs(g) / nu))
        hist.append(err)
        if verbose:
            print(f"newton it={it} err={err:.3e} K={ev['K']:.15e}")
        if err <= tol:
            break
        if it >= maxit:
            raise RuntimeError(f"oracle Newton did not converge: err={err}")
        delta = _newton_direction(ev["L"], g)
        gn = np.linalg.norm(g)
        alpha = 1.0
        while True:
            trial = psi + alpha * delta
            et = laguerre(pos, trial, box, nu, mode)
            n_eval += 1
            if et["vol"].min() >= eps0 and np.linalg.norm(et["grad"]) <= (1 - alpha / 2) * gn:
                break
            alpha *= 0.5
            if alpha < 2.0 ** -30:
                raise RuntimeError("oracle line search found no descent")
        # the gauge shift leaves every cell unchanged (all planes depend on psi_i - psi_j)
        psi = trial - trial.mean()
        ev = et
        it += 1
    disp = displacement(ev)
    return psi, dict(vol=ev["vol"], centroid=ev["centroid"], disp=disp, it=it,
                     n_eval=n_eval, hist=hist, K=ev["K"], L=ev["L"])


def displacement(ev):
    """Zel'dovich displacement of cell i: y_i - centroid(V_i), minimum image.

    In local coordinates this is minus the local centroid, which already lies
    within half a box of the seed.
    """
    return -ev["local_centroid"]


def potential_mesh(pos, psi, box, M):
    """phi_I at the M^3 mesh points (m + 1/2) L / M, and the cell i(q) containing each
    (the Legendre transform of psi, Sec. "Monge-Ampere-Kantorovich Reconstruction").
    Returns (phi[M, M, M], owner[M, M, M]) indexed [z, y, x]."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    L = _box(box)
    phi = np.empty(M ** 3)
    owner = np.empty(M ** 3, dtype=np.int64)
    if lib.oracle_potential_mesh(pos.shape[0], _ptr(pos), _ptr(psi), _ptr(L), M, _ptr(phi),
                                 _ptr(owner)) != 0:
        raise ValueError("M must be >= 1")
    return phi.reshape(M, M, M), owner.reshape(M, M, M)


def deposit(pos, psi, box, M, lam, mass=None):
    """Mass density on the M^3 mesh of the cells moved by the Zel'dovich map
    q -> q + lam (x_i - q) (each cell shrunk about its point by 1 - lam, its mass spread
    uniformly), by exact clipping with the voxels (last paragraph of Sec.
    "Monge-Ampere-Kantorovich Reconstruction", Fig. 1). Indexed [z, y, x]."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    L = _box(box)
    N = pos.shape[0]
    if mass is None:
        mass = np.full(N, float(np.prod(L)) / N)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    rho = np.empty(M ** 3)
    rc = lib.oracle_deposit(N, _ptr(pos), _ptr(psi), _ptr(mass), _ptr(L), M, float(lam),
                            _ptr(rho))
    if rc == -1:
        raise ValueError("need M >= 1 and 0 <= lam < 1")
    if rc == -2:
        raise RuntimeError("oracle polytope capacity exceeded")
    return rho.reshape(M, M, M)


def power_spectrum(rho, L, nbins=None):
    """Power spectrum of the density contrast of a periodic M^3 mesh: the estimator
    behind the fractional BAO signal d(k) = P_wig(k)/P_nw(k) - 1 (Sec. "BAO
    reconstruction", Fig. 2).

    delta = rho / mean(rho) - 1; delta_k = (sum_x delta(x) e^{-i k.x}) / M^3 over the
    full complex FFT, k = 2 pi n / L with n the integer frequencies of numpy's fftfreq;
    P(k) = L^3 |delta_k|^2. Mode n != 0 goes into bin b = floor(|n| + 1/2), kept for
    1 <= b <= nbins (default M // 2). Returns (P, kmean, nmodes): per bin the mean P over
    its modes, their mean |k|, and their count.
    """
    rho = np.asarray(rho, dtype=np.float64)
    M = rho.shape[0]
    assert rho.shape == (M, M, M)
    if nbins is None:
        nbins = M // 2
    delta = rho / rho.mean() - 1.0
    dk = np.fft.fftn(delta) / M ** 3
    p = float(L) ** 3 * np.abs(dk) ** 2
    n = np.fft.fftfreq(M, d=1.0 / M)
    nz, ny, nx = np.meshgrid(n, n, n, indexing="ij")
    nn = np.sqrt(nx * nx + ny * ny + nz * nz)
    b = np.floor(nn + 0.5).astype(np.int64)
    sel = (b >= 1) & (b <= nbins)
    cnt = np.bincount(b[sel], minlength=nbins + 1)[1:]
    psum = np.bincount(b[sel], weights=p[sel], minlength=nbins + 1)[1:]
    ksum = np.bincount(b[sel], weights=nn[sel], minlength=nbins + 1)[1:]
    with np.errstate(invalid="ignore", divide="ignore"):
        P = np.where(cnt > 0, psum / cnt, 0.0)
        kmean = np.where(cnt > 0, 2.0 * np.pi / float(L) * ksum / cnt, 0.0)
    return P, kmean, cnt
