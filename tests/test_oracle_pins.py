"""Pins for the CPU oracle against facts fixed by the mathematics (no GPU).

The paper (arXiv:2110.08868) prints no worked example, so the oracle is pinned by
closed forms (lattice, translated lattice, two-seed slab, separable plane wave),
brute force, finite differences of K (eq. SDK), invariants of the Laguerre
diagram (eq. laguerrecell), an independent point-location estimate and a
library kNN.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import sdot_oracle as O
from paper_2110_08868_gb300 import ics


def _lattice_expect(n, L):
    a = L / n
    return a, a ** 3


@pytest.mark.parametrize("n", [4, 5])
@pytest.mark.parametrize("mode", ["brute", "certified"])
def test_lattice_cubes(n, mode):
    # psi = 0 on a lattice: every cell is the cube of side a around its seed;
    # facets are the 6 face neighbours with area a^2 at distance a, so
    # L = a * (7-point Laplacian); K = N a^5 / 8 (int over cube of 1/2|p|^2).
    L = 1.0
    q = ics.lattice(n, L)
    N = n ** 3
    a, v = _lattice_expect(n, L)
    nu = ics.uniform_masses(N, L)
    ev = O.laguerre(q, np.zeros(N), L, nu, mode=mode)
    np.testing.assert_allclose(ev["vol"], v, rtol=1e-13)
    np.testing.assert_allclose(ev["local_centroid"], 0.0, atol=1e-14)
    assert abs(ev["K"] - N * a ** 5 / 8) < 1e-13 * N * a ** 5
    Lm = ev["L"].toarray()
    np.testing.assert_allclose(np.diag(Lm), 6 * a, rtol=1e-13)
    off = Lm - np.diag(np.diag(Lm))
    # each row: exactly 6 entries equal to -a (n >= 3 so the 6 are distinct)
    for i in range(N):
        nz = off[i][np.abs(off[i]) > 1e-12 * a]
        assert nz.size == 6
        np.testing.assert_allclose(nz, -a, rtol=1e-12)
    np.testing.assert_allclose(O.displacement(ev), 0.0, atol=1e-14)


def test_translated_lattice():
    # y = q + t: psi = 0 already balances the masses; cells are cubes centred on
    # the seeds, so the displacement is 0 (a uniform shift is invisible on a torus).
    n, L = 4, 1.0
    t = np.array([0.013, -0.071, 0.2])
    y = np.mod(ics.lattice(n, L) + t, L)
    N = n ** 3
    ev = O.laguerre(y, np.zeros(N), L, ics.uniform_masses(N, L))
    np.testing.assert_allclose(ev["vol"], (L / n) ** 3, rtol=1e-13)
    np.testing.assert_allclose(O.displacement(ev), 0.0, atol=1e-14)


@pytest.mark.parametrize("delta", [0.0, 0.01, -0.03])
def test_two_seed_slab(delta):
    # seeds (1/4,1/2,1/2) and (3/4,1/2,1/2), psi = (delta, 0): the two facets with the
    # images of seed 2 at x = 1/4 + 1/4 + 2 delta and x = 1/4 - 1/4 - 2 delta, so
    # V_1 = 1/2 + 4 delta; each facet has area 1 and |d| = 1/2, so L_12 = -4.
    y = np.array([[0.25, 0.5, 0.5], [0.75, 0.5, 0.5]])
    psi = np.array([delta, 0.0])
    for mode in ("brute", "certified"):
        ev = O.laguerre(y, psi, 1.0, np.array([0.5, 0.5]), mode=mode)
        assert abs(ev["vol"][0] - (0.5 + 4 * delta)) < 1e-14
        assert abs(ev["vol"][1] - (0.5 - 4 * delta)) < 1e-14
        Lm = ev["L"].toarray()
        assert abs(Lm[0, 1] + 4.0) < 1e-13 and abs(Lm[1, 0] + 4.0) < 1e-13
        assert abs(Lm[0, 0] - 4.0) < 1e-13


@pytest.mark.parametrize("f", [0.3, 0.5, 0.62])
def test_two_seed_unequal_masses_solve(f):
    # masses (f, 1 - f) of the unit box for the slab pair above: V_1 = 1/2 + 4 delta must
    # equal f, so psi_1 - psi_2 = (f - 1/2) / 4; cell 1 spans x in [-2 delta, 1/2 + 2 delta],
    # symmetric about its seed (and cell 2 about its own), so both displacements vanish
    y = np.array([[0.25, 0.5, 0.5], [0.75, 0.5, 0.5]])
    psi, info = O.solve(y, np.array([f, 1.0 - f]), 1.0, tol=1e-13)
    assert abs((psi[0] - psi[1]) - (f - 0.5) / 4) < 1e-13
    assert abs(psi.sum()) < 1e-15
    np.testing.assert_allclose(info["vol"], [f, 1.0 - f], rtol=0, atol=1e-13)
    np.testing.assert_allclose(info["disp"], 0.0, atol=1e-13)


def plane_wave(n, L, amps, phases):
    """Separable displacement s_a(q_a) = A_a sin(2 pi q_a / L + phi_a) and its exact psi.

    With 1 + s' > 0 (no shell crossing) and zero lattice mean, the power distance
    separates per axis and every Laguerre cell is the lattice cube of its seed. The
    1D weights follow from equal power at the cube face p = q_m + a/2:
      psi_{m+1} - psi_m = 1/2 D^2 - D (p - x_m),  D = x_{m+1} - x_m (unwrapped).
    """
    a = L / n
    g = (np.arange(n) + 0.5) * a
    psis, xs = [], []
    for A, ph in zip(amps, phases):
        assert 2 * np.pi * A / L < 1
        x = g + A * np.sin(2 * np.pi * g / L + ph)
        xn = np.append(x, x[0] + L)
        p = g + 0.5 * a
        D = np.diff(xn)
        inc = 0.5 * D ** 2 - D * (p - x)
        assert abs(inc.sum()) < 1e-12 * L * L  # closes around the torus
        psis.append(np.concatenate([[0.0], np.cumsum(inc[:-1])]))
        xs.append(x)
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    y = np.stack([xs[0][ix], xs[1][iy], xs[2][iz]], axis=1)
    psi = psis[0][ix] + psis[1][iy] + psis[2][iz]
    s = y - ics.lattice(n, L)
    return np.mod(y, L), psi - psi.mean(), s


def test_plane_wave_closed_form_cells():
    n, L = 6, 1.0
    y, psi, s = plane_wave(n, L, [0.09, 0.05, 0.12], [0.3, 1.1, -0.4])
    N = n ** 3
    ev = O.laguerre(y, psi, L, ics.uniform_masses(N, L))
    np.testing.assert_allclose(ev["vol"], (L / n) ** 3, rtol=1e-11)
    np.testing.assert_allclose(O.displacement(ev), s, atol=1e-11 * L / n)


def test_plane_wave_newton_recovers_closed_form():
    n, L = 6, 1.0
    y, psi_exact, s = plane_wave(n, L, [0.09, 0.05, 0.12], [0.3, 1.1, -0.4])
    N = n ** 3
    nu = ics.uniform_masses(N, L)
    psi, info = O.solve(y, nu, L, tol=1e-12)
    a = L / n
    np.testing.assert_allclose(psi, psi_exact, atol=1e-9 * a * a)
    np.testing.assert_allclose(info["disp"], s, atol=1e-9 * a)


def _random_case(n=5, L=1.0, rms=0.3, seed=7, psi_scale=0.01):
    y, _, _ = ics.zeldovich_box(n, L, ics.spectrum_kinv, rms, seed)
    a = L / n
    rng = np.random.default_rng(seed + 1)
    psi = psi_scale * a * a * rng.standard_normal(y.shape[0])
    return y, psi, L


def test_brute_equals_certified():
    for seed in (3, 4):
        y, psi, L = _random_case(n=6, seed=seed)
        b = O.cells(y, psi, L, "brute")
        c = O.cells(y, psi, L, "certified")
        np.testing.assert_allclose(b["vol"], c["vol"], rtol=1e-12, atol=0)
        np.testing.assert_allclose(b["m1"], c["m1"], atol=1e-15)
        Lb = O.hessian_laplacian(b, y.shape[0]).toarray()
        Lc = O.hessian_laplacian(c, y.shape[0]).toarray()
        np.testing.assert_allclose(Lb, Lc, atol=1e-12 * np.abs(Lb).max())


def test_brute_equals_certified_at_solved_clumpy_psi():
    # psi of an oracle-solved clumpy box spreads over ~5 a^2 (the regime of the
    # 256^3 + clumps workload, whose solved psi spreads over several a^2), so the
    # certificate's psi term R + sqrt(R^2 + 2 (psi_max - psi_i)) decides where the
    # certified cells stop
    n, L = 7, 1.0
    a = L / n
    y, _, _ = ics.zeldovich_box(n, L, ics.spectrum_kinv, 0.3, 5)
    y = np.ascontiguousarray(ics.add_clumps(y, L, n, 1, 120, 0.05, 6))
    N = y.shape[0]
    psi, info = O.solve(y, ics.uniform_masses(N, L), L, tol=1e-10)
    assert (psi.max() - psi.min()) > 4.0 * a * a
    b = O.cells(y, psi, L, "brute")
    c = O.cells(y, psi, L, "certified")
    np.testing.assert_allclose(b["vol"], c["vol"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(b["m1"], c["m1"], atol=1e-14 * a ** 4)
    Lb = O.hessian_laplacian(b, N).toarray()
    Lc = O.hessian_laplacian(c, N).toarray()
    np.testing.assert_allclose(Lb, Lc, atol=1e-12 * np.abs(Lb).max())


@pytest.mark.parametrize("n,dist,dpsi", [(5, 2, 1.5), (7, 3, 3.75)])
@pytest.mark.parametrize("mode", ["brute", "certified"])
def test_hidden_heavy_neighbour_closed_form(n, dist, dpsi, mode):
    # Lattice, psi = 0 except psi_j = dpsi a^2 for the seed j that sits `dist` spacings
    # along +x from seed i. Its bisector with i, p_x <= (dist^2 a^2 / 2 - dpsi a^2) /
    # (dist a) = a/4, cuts the cube cell of i although j is no face neighbour, and j's
    # image on the other side (n - dist spacings away) does not reach it. So
    # V_i = 3/4 a^3 and the local centroid is (-a/8, 0, 0). A certificate without the
    # psi term (2R = sqrt(3) a) stops before j in both cases; one with half the psi term
    # (R + sqrt(R^2 + dpsi)) stops before j in the (7, 3) case.
    L = 1.0
    a = L / n
    y = ics.lattice(n, L)
    N = n ** 3
    i = (n // 2) * (1 + n + n * n) - dist // 2  # an interior seed; j = i + dist along x
    j = i + dist
    assert np.isclose(y[j, 0] - y[i, 0], dist * a)
    psi = np.zeros(N)
    psi[j] = dpsi * a * a
    c = O.cells(y, psi, L, mode, idx=np.array([i]))
    np.testing.assert_allclose(c["vol"][0], 0.75 * a ** 3, rtol=1e-12)
    np.testing.assert_allclose(c["m1"][0] / c["vol"][0], [-a / 8, 0.0, 0.0], atol=1e-13 * a)
    assert j in set(c["fj"][0, :c["nfac"][0]].tolist())


def test_invariants():
    y, psi, L = _random_case(n=6, seed=11)
    N = y.shape[0]
    nu = ics.uniform_masses(N, L)
    ev = O.laguerre(y, psi, L, nu)
    assert ev["vol"].min() > 0.01 * nu[0]  # no empty cell
    # volumes tile the box
    assert abs(ev["vol"].sum() - L ** 3) < 1e-12 * L ** 3
    Lm = ev["L"].toarray()
    # symmetric, zero row sums, positive semi-definite with a 1-D kernel
    np.testing.assert_allclose(Lm, Lm.T, atol=1e-12 * np.abs(Lm).max())
    np.testing.assert_allclose(Lm.sum(axis=1), 0.0, atol=1e-12 * np.abs(Lm).max())
    w = np.linalg.eigvalsh(Lm)
    assert w[0] > -1e-10 * w[-1] and w[1] > 1e-8 * w[-1]
    # psi + c changes no cell
    ev2 = O.laguerre(y, psi + 0.123, L, nu)
    np.testing.assert_allclose(ev2["vol"], ev["vol"], rtol=1e-12)
    # permutation equivariance
    perm = np.random.default_rng(0).permutation(N)
    ev3 = O.laguerre(y[perm], psi[perm], L, nu[perm])
    np.testing.assert_allclose(ev3["vol"], ev["vol"][perm], rtol=1e-12)
    # translation covariance (positions shifted on the torus, same cells)
    t = np.array([0.31, -0.17, 0.05])
    ev4 = O.laguerre(np.mod(y + t, L), psi, L, nu)
    np.testing.assert_allclose(ev4["vol"], ev["vol"], rtol=1e-12)
    np.testing.assert_allclose(ev4["local_centroid"], ev["local_centroid"], atol=1e-13)


def test_finite_differences():
    # dK/dpsi_i = nu_i - V_i and dV_i/dpsi_j = L_ij (eq. SDK differentiated)
    y, psi, L = _random_case(n=5, seed=21)
    N = y.shape[0]
    nu = ics.uniform_masses(N, L)
    a = L / 5
    ev = O.laguerre(y, psi, L, nu)
    Lm = ev["L"].toarray()
    h = 1e-6 * a * a
    rng = np.random.default_rng(5)
    for i in rng.choice(N, 6, replace=False):
        e = np.zeros(N)
        e[i] = h
        p = O.laguerre(y, psi + e, L, nu, with_hessian=False)
        m = O.laguerre(y, psi - e, L, nu, with_hessian=False)
        g_fd = (p["K"] - m["K"]) / (2 * h)
        assert abs(g_fd - ev["grad"][i]) < 1e-6 * nu[i]
        col_fd = (p["vol"] - m["vol"]) / (2 * h)
        np.testing.assert_allclose(col_fd, Lm[:, i], atol=1e-6 * np.abs(Lm[i, i]))


def test_point_location_volumes_and_centroids():
    # Independent of the polytope code: assign a fine grid of sample points to the
    # cell minimising 1/2|q - y_j|^2 - psi_j (min image) and compare volume and
    # centroid estimates with the clipped cells.
    n, L = 3, 1.0
    a = L / n
    rng = np.random.default_rng(31)
    y = np.mod(ics.lattice(n, L) + rng.uniform(-0.25, 0.25, (n ** 3, 3)) * a, L)
    psi = 0.1 * a * a * rng.standard_normal(n ** 3)
    N = y.shape[0]
    m = 72
    g = (np.arange(m) + 0.5) / m * L
    Q = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    best = np.full(Q.shape[0], np.inf)
    arg = np.zeros(Q.shape[0], dtype=np.int64)
    off = np.zeros((Q.shape[0], 3))
    for j in range(N):
        d = Q - y[j]
        d -= L * np.round(d / L)
        pw = 0.5 * np.sum(d * d, axis=1) - psi[j]
        better = pw < best
        best[better] = pw[better]
        arg[better] = j
        off[better] = d[better]
    ev = O.laguerre(y, psi, L)
    cnt = np.bincount(arg, minlength=N)
    vol_pl = cnt / Q.shape[0] * L ** 3
    assert ev["vol"].min() > 0.1 * L ** 3 / N
    np.testing.assert_allclose(vol_pl, ev["vol"], rtol=0.03)
    for j in range(N):
        cen = off[arg == j].mean(axis=0)
        np.testing.assert_allclose(cen, ev["local_centroid"][j], atol=0.02 * L / n)


def test_knn_against_kdtree():
    rng = np.random.default_rng(2)
    L = 1.0
    y = rng.uniform(0, L, size=(700, 3))
    k = 24
    nb, d2 = O.knn(y, L, k)
    tree = cKDTree(y, boxsize=L)
    dd, ii = tree.query(y, k=k + 1)
    np.testing.assert_array_equal(nb, ii[:, 1:])
    np.testing.assert_allclose(np.sqrt(d2), dd[:, 1:], rtol=1e-13)


def test_knn_lattice_tie_order():
    # 4^3 lattice: 6 face neighbours (d^2 = a^2), then 12 edge (2a^2), 8 corner (3a^2),
    # then the 3 half-box neighbours (d^2 = 4a^2, counted once each); ties by index.
    n, L = 4, 1.0
    y = ics.lattice(n, L)
    nb, d2 = O.knn(y, L, 29)
    for i in (0, 21, 63):
        ix, iy, iz = i % n, (i // n) % n, i // (n * n)
        groups = {}
        for j in range(n ** 3):
            if j == i:
                continue
            jx, jy, jz = j % n, (j // n) % n, j // (n * n)
            dd = [min((jx - ix) % n, (ix - jx) % n), min((jy - iy) % n, (iy - jy) % n),
                  min((jz - iz) % n, (iz - jz) % n)]
            groups.setdefault(sum(c * c for c in dd), []).append(j)
        expect = []
        for key in sorted(groups):
            expect += sorted(groups[key])
        assert list(nb[i]) == expect[:29]


def test_newton_c1_small_converges():
    y, nu, L = ics.make_config(**ics.CONFIGS["zeldovich-16^3-kinv-0.3a"])
    # a 8^3 version of the same recipe keeps the CPU suite fast
    y, _, _ = ics.zeldovich_box(8, 1.0, ics.spectrum_kinv, 0.3, 1)
    N = y.shape[0]
    nu = ics.uniform_masses(N, 1.0)
    psi, info = O.solve(y, nu, 1.0, tol=1e-10)
    assert info["hist"][-1] <= 1e-10
    assert abs(psi.sum()) < 1e-12
    np.testing.assert_allclose(info["vol"], nu, rtol=1e-10)


# --- phi_I on a mesh, the Zel'dovich move and the Eulerian deposit ----------------------

def test_potential_lattice_closed_form():
    # psi = 0 on a lattice: phi_I(q) = 1/2 |q - nearest lattice point|^2
    n, L, M = 4, 1.0, 8
    a = L / n
    phi, owner = O.potential_mesh(ics.lattice(n, L), np.zeros(n ** 3), L, M)
    g = (np.arange(M) + 0.5) * L / M
    off = (g - (np.floor(g / a) + 0.5) * a) ** 2  # squared offset per axis
    expect = 0.5 * (off[:, None, None] + off[None, :, None] + off[None, None, :])
    np.testing.assert_allclose(phi, expect, rtol=1e-14)
    c = np.floor(g / a).astype(int)
    np.testing.assert_array_equal(owner, c[None, None, :] + n * c[None, :, None]
                                  + n * n * c[:, None, None])


def test_potential_plane_wave_closed_form():
    # separable plane wave: the cells are the lattice cubes, so the owner of q is the
    # cube containing it and phi_I(q) = 1/2 |q - y_j|^2 - psi_j (no mesh point lies on a
    # cube face for n = 5, M = 12)
    n, L, M = 5, 1.0, 12
    a = L / n
    y, psi, _ = plane_wave(n, L, [0.03, 0.02, 0.035], [0.3, 1.1, -0.4])
    phi, owner = O.potential_mesh(y, psi, L, M)
    g = (np.arange(M) + 0.5) * L / M
    c = np.floor(g / a).astype(int)
    j = c[None, None, :] + n * c[None, :, None] + n * n * c[:, None, None]
    np.testing.assert_array_equal(owner, j)
    q = np.stack(np.meshgrid(g, g, g, indexing="ij")[::-1], -1)  # [z, y, x, (x, y, z)]
    d = q - y[j]
    d -= L * np.round(d / L)
    np.testing.assert_allclose(phi, 0.5 * (d ** 2).sum(-1) - psi[j], rtol=0, atol=1e-14)


def _overlap_1d(c, w, M, L):
    """fraction of each interval [c_i - w/2, c_i + w/2] (periodic) in each of M bins"""
    h = L / M
    out = np.zeros((c.size, M))
    for i, ci in enumerate(c):
        lo, hi = ci - 0.5 * w, ci + 0.5 * w
        for v in range(int(np.floor(lo / h)), int(np.floor(hi / h)) + 1):
            ov = min(hi, (v + 1) * h) - max(lo, v * h)
            if ov > 0:
                out[i, v % M] += ov / w
    return out


@pytest.mark.parametrize("lam,M", [(0.0, 5), (0.3, 9), (0.7, 12)])
def test_deposit_plane_wave_closed_form(lam, M):
    # the cells of the separable plane wave are the lattice cubes; moved by the
    # Zel'dovich map each becomes a cube of side (1 - lam) a centred at q + lam s(q), so
    # the voxel masses are products of 1-D interval overlaps
    n, L = 5, 1.0
    a = L / n
    amps, phases = [0.03, 0.02, 0.035], [0.3, 1.1, -0.4]
    y, psi, s = plane_wave(n, L, amps, phases)
    rho = O.deposit(y, psi, L, M, lam)
    g = (np.arange(n) + 0.5) * a
    w = (1 - lam) * a
    ov = []
    for ax, (A, ph) in enumerate(zip(amps, phases)):
        c = g + lam * A * np.sin(2 * np.pi * g / L + ph)
        ov.append(_overlap_1d(c, w, M, L).sum(axis=0))
    nu, vox = a ** 3, (L / M) ** 3
    expect = nu / vox * ov[2][:, None, None] * ov[1][None, :, None] * ov[0][None, None, :]
    np.testing.assert_allclose(rho, expect, rtol=1e-11, atol=1e-12)


def test_deposit_conserves_mass_and_is_uniform_at_the_solution():
    # any psi: the deposited masses sum to the seeds' masses; at the OT solution and
    # lam = 0 every cell has volume nu_i, so the density is 1 everywhere
    n, L, M = 5, 1.0, 7
    y, _, _ = ics.zeldovich_box(n, L, ics.spectrum_kinv, 0.3, 12)
    N = y.shape[0]
    nu = ics.uniform_masses(N, L)
    psi = 0.05 * (L / n) ** 2 * np.random.default_rng(3).standard_normal(N)
    for lam in (0.0, 0.4):
        rho = O.deposit(y, psi, L, M, lam)
        assert abs(rho.sum() * (L / M) ** 3 - nu.sum()) < 1e-12 * L ** 3
    psi_s, _ = O.solve(y, nu, L, tol=1e-12)
    np.testing.assert_allclose(O.deposit(y, psi_s, L, M, 0.0), 1.0, rtol=0, atol=1e-10)


# --- power spectrum of a mesh (the estimator behind d(k), Sec. "BAO reconstruction") ---

def test_power_spectrum_parseval():
    # with every mode binned, sum_b nmodes_b P_b / L^3 = mean(delta^2) (Parseval)
    rng = np.random.default_rng(21)
    M, L = 8, 3.0
    rho = 1.0 + 0.1 * rng.standard_normal((M, M, M))
    P, _, cnt = O.power_spectrum(rho, L, nbins=8)
    delta = rho / rho.mean() - 1.0
    assert cnt.sum() == M ** 3 - 1
    assert abs((cnt * P).sum() / L ** 3 - (delta * delta).mean()) <= 1e-14


def test_power_spectrum_brute_force_dft():
    # explicit sums over the mesh points for every mode of a 4^3 mesh
    rng = np.random.default_rng(22)
    M, L = 4, 2.0
    rho = 1.0 + 0.2 * rng.uniform(-1, 1, (M, M, M))
    delta = rho / rho.mean() - 1.0
    n1 = [0, 1, -2, -1]
    psum = np.zeros(5)
    cnt = np.zeros(5, dtype=int)
    ksum = np.zeros(5)
    for nz in n1:
        for ny in n1:
            for nx in n1:
                s = 0j
                for z in range(M):
                    for y in range(M):
                        for x in range(M):
                            s += delta[z, y, x] * np.exp(-2j * np.pi * (nx * x + ny * y + nz * z) / M)
                nn = np.sqrt(nx * nx + ny * ny + nz * nz)
                b = int(np.floor(nn + 0.5))
                if 1 <= b <= 4:
                    psum[b] += L ** 3 * abs(s / M ** 3) ** 2
                    cnt[b] += 1
                    ksum[b] += 2 * np.pi / L * nn
    P, k, c = O.power_spectrum(rho, L, nbins=4)
    np.testing.assert_array_equal(c, cnt[1:])
    assert cnt[4] == 0 and P[3] == 0.0  # |n| <= sqrt(12) < 3.5 on a 4^3 mesh
    np.testing.assert_allclose(P[:3], psum[1:4] / cnt[1:4], rtol=1e-12)
    np.testing.assert_allclose(k[:3], ksum[1:4] / cnt[1:4], rtol=1e-14)


def test_power_spectrum_plane_wave():
    # delta = A cos(2 pi 3 x / L): the two modes +-(3, 0, 0) hold (A/2)^2 each, nothing else
    M, L, A = 16, 5.0, 0.3
    x = (np.arange(M) + 0.5) * L / M
    rho = np.broadcast_to(1.0 + A * np.cos(2 * np.pi * 3 * x / L), (M, M, M)).copy()
    P, _, cnt = O.power_spectrum(rho, L)
    expect = np.zeros(M // 2)
    expect[2] = 2 * L ** 3 * (A / 2) ** 2 / cnt[2]
    np.testing.assert_allclose(P, expect, rtol=1e-12, atol=1e-25)


def test_power_spectrum_bin_counts():
    # bin b holds the lattice points n with b - 1/2 <= |n| < b + 1/2: bin 1 is |n|^2 in
    # {1, 2} (6 + 12 points), bin 2 is |n|^2 in {3, 4, 5, 6} (8 + 6 + 24 + 24)
    _, _, cnt = O.power_spectrum(np.ones((8, 8, 8)) + 1e-3, 1.0)
    assert cnt[0] == 18 and cnt[1] == 62
