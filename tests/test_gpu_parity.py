"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (from the arithmetic, stated here once):
  * kNN lists: bit-exact (integer result of an exact FP64 key).
  * FP64 volumes / centroids: 1e-10 relative (to a^3 / a); Hessian entries 1e-10 of the
    row diagonal.
  * Mixed precision (FP32 geometry in units of the spacing a, FP64 sums): volumes 2e-5
    relative, centroids and displacements 2e-5 a; Hessian entries 1e-4 of the row
    diagonal plus 1e-6 of the mean diagonal: FP32 vertex coordinates carry an absolute
    error of about 1e-7 a, so the facets of a nearly empty cell (a random psi empties
    some) have an absolute error at that floor, which is large next to the cell's own
    tiny diagonal; the solve reaches the same max|V - nu|/nu criterion.
  * Displacement at convergence (both sides solved to 1e-10): 1e-6 a.
"""
import numpy as np
import pytest

import sdot_oracle as O
from paper_2110_08868_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2110_08868_gb300 import binding as B  # noqa: E402


def c1():
    return ics.make_config(**ics.CONFIGS["zeldovich-16^3-kinv-0.3a"])


def _hess_close(Lg, Lo, tol, floor=0.0):
    """Every entry within tol of its row's diagonal plus floor of the mean diagonal
    (rows of empty cells, with a zero diagonal, use the mean). Returns (ok, worst ratio
    of the error to that bound, scaled to tol)."""
    Lg = Lg.toarray() if hasattr(Lg, "toarray") else Lg
    Lo = Lo.toarray() if hasattr(Lo, "toarray") else Lo
    d = np.abs(np.diag(Lo))
    bound = (tol * np.where(d > 0, d, d.mean()) + floor * d.mean())[:, None]
    r = np.max(np.abs(Lg - Lo) / bound)
    return r <= 1.0, r * tol


def test_knn_bit_exact_c1():
    y, nu, L = c1()
    s = B.Solver(y, [L] * 3, precision="fp64")
    nb = s.knn()
    ref, _ = O.knn(y, L, 24)
    np.testing.assert_array_equal(nb, ref)


@pytest.mark.parametrize("k", [8, 24, 33])
def test_knn_bit_exact_ties_and_ragged(k):
    # 7^3 lattice (many exact ties) plus 17 extra random points (ragged N)
    rng = np.random.default_rng(4)
    q = ics.lattice(7, 1.0)
    y = np.concatenate([q, rng.uniform(0, 1, (17, 3))])
    s = B.Solver(y, [1.0] * 3, precision="fp64", k=k)
    ref, _ = O.knn(y, 1.0, k)
    np.testing.assert_array_equal(s.knn(), ref)


@pytest.mark.parametrize("prec,vtol,ctol,htol,hfloor", [("fp64", 1e-10, 1e-10, 1e-10, 0.0),
                                                         ("mixed", 2e-5, 2e-5, 1e-4, 1e-6)])
def test_laguerre_psi0_c1(prec, vtol, ctol, htol, hfloor):
    y, nu, L = c1()
    N = y.shape[0]
    a = L / 16
    s = B.Solver(y, [L] * 3, precision=prec)
    g = s.laguerre(with_hessian=True)
    o = O.laguerre(y, np.zeros(N), L, nu)
    np.testing.assert_allclose(g["vol"], o["vol"], rtol=0, atol=vtol * a ** 3)
    dc = g["centroid"] - o["centroid"]
    dc -= L * np.round(dc / L)
    assert np.max(np.abs(dc)) <= ctol * a
    ok, err = _hess_close(g["hess"], o["L"], htol, hfloor)
    assert ok, err


@pytest.mark.parametrize("prec,vtol,htol,hfloor", [("fp64", 1e-10, 1e-10, 0.0),
                                                   ("mixed", 2e-5, 1e-4, 1e-6)])
def test_laguerre_random_psi_c1(prec, vtol, htol, hfloor):
    # a random psi makes the cells leave their seeds: the security test of the first
    # pass finds cutters beyond the k nearest seeds and re-queues those cells, whose
    # second pass must match the oracle like every other cell
    y, nu, L = c1()
    N = y.shape[0]
    a = L / 16
    rng = np.random.default_rng(9)
    psi = 0.2 * a * a * rng.standard_normal(N)
    s = B.Solver(y, [L] * 3, precision=prec)
    g = s.laguerre(psi, with_hessian=True, allow_empty=True)
    requeued = np.flatnonzero(s.status() & 8)
    assert requeued.size > 0, "the re-queue pass did not run"
    o = O.laguerre(y, psi, L, nu)
    np.testing.assert_allclose(g["vol"], o["vol"], rtol=0, atol=vtol * a ** 3)
    np.testing.assert_allclose(g["vol"][requeued], o["vol"][requeued], rtol=0,
                               atol=vtol * a ** 3)
    ok, err = _hess_close(g["hess"], o["L"], htol, hfloor)
    assert ok, err


def hub_box(n_sphere=60, seed=5):
    """A 10^3 lattice whose central point is replaced by a hub seed with n_sphere seeds on
    a sphere of radius 0.4 a around it: the hub's cell has n_sphere faces (every
    bisector with a point of the sphere is tangent to the sphere of radius 0.2 a),
    more than the small polytope of the first passes holds."""
    n, L = 10, 1.0
    a = L / n
    q = ics.lattice(n, L)
    rng = np.random.default_rng(seed)
    q = np.mod(q + rng.uniform(-0.1, 0.1, q.shape) * a, L)
    c = np.array([0.5, 0.5, 0.5])
    d = q - c
    d -= L * np.round(d / L)
    keep = np.linalg.norm(d, axis=1) > 0.6 * a
    k = np.arange(n_sphere) + 0.5
    th = np.arccos(1 - 2 * k / n_sphere)
    ph = np.pi * (1 + 5 ** 0.5) * k
    sph = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    y = np.concatenate([q[keep], c[None], c + 0.4 * a * sph])
    return np.ascontiguousarray(y), L, int(keep.sum())


@pytest.mark.parametrize("prec,vtol,ctol", [("fp64", 1e-10, 1e-10), ("mixed", 2e-5, 2e-5)])
def test_hub_cell_goes_through_the_large_polytope(prec, vtol, ctol):
    # the hub overflows the small polytope of the first two passes, so the third pass
    # clips it again in FP64 with the large one; every cell must match the oracle
    y, L, hub = hub_box()
    N = y.shape[0]
    a = L / 10
    nu = ics.uniform_masses(N, L)
    s = B.Solver(y, [L] * 3, precision=prec)
    g = s.laguerre(None, allow_empty=True)
    st = s.status()
    assert st[hub] & (32 | 64), ("the large-polytope re-clip did not run", int(st[hub]))
    assert not (st & 2).any()
    o = O.laguerre(y, np.zeros(N), L, nu, with_hessian=False)
    np.testing.assert_allclose(g["vol"], o["vol"], rtol=0, atol=vtol * a ** 3)
    dc = g["centroid"] - o["centroid"]
    dc -= L * np.round(dc / L)
    assert np.max(np.abs(dc)) <= ctol * a
    assert int(o["cells"]["nfac"][hub]) == 60


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hessian_exactly_symmetric_zero_rowsum(prec):
    # after a few warm-started evaluations at moving psi (the solve's access pattern)
    y, nu, L = c1()
    N = y.shape[0]
    a = L / 16
    s = B.Solver(y, [L] * 3, precision=prec)
    rng = np.random.default_rng(3)
    for step in range(4):
        g = s.laguerre(0.05 * step * a * a * rng.standard_normal(N), with_hessian=True,
                       allow_empty=True)
        H = g["hess"]
        assert abs(H - H.T).max() == 0.0
        assert np.abs(np.asarray(H.sum(axis=1))).max() <= 1e-12 * H.diagonal().max()
        assert (H.diagonal() >= 0).all()
        off = H - __import__("scipy.sparse", fromlist=["diags"]).diags(H.diagonal())
        assert off.max() <= 0.0


def test_solve_fp64_matches_oracle_displacement():
    y, nu, L = c1()
    a = L / 16
    s = B.Solver(y, [L] * 3, precision="fp64")
    st = s.solve(1e-10)
    assert st["max_rel_err"] <= 1e-10
    psi_o, info = O.solve(y, nu, L, tol=1e-11)
    d = s.displacement()
    assert np.max(np.abs(d - info["disp"])) <= 1e-6 * a
    np.testing.assert_allclose(s.psi(), psi_o, atol=1e-7 * a * a)


def test_solve_mixed_reaches_criterion():
    y, nu, L = c1()
    a = L / 16
    s = B.Solver(y, [L] * 3, precision="mixed")
    st = s.solve(1e-4)
    assert st["max_rel_err"] <= 1e-4
    _, info = O.solve(y, nu, L, tol=1e-11)
    err = np.max(np.abs(s.displacement() - info["disp"])) / a
    # a 1e-4 volume stop leaves centroid errors of order 1e-5 a
    assert err < 1e-3, err


def test_lattice_zero_iterations():
    n, L = 12, 3.0
    y = ics.lattice(n, L)
    s = B.Solver(y, [L] * 3, precision="fp64")
    st = s.solve(1e-12)
    assert st["newton_iters"] == 0
    np.testing.assert_allclose(s.displacement(), 0.0, atol=1e-12 * L / n)


def test_plane_wave_closed_form_gpu():
    from test_oracle_pins import plane_wave

    # amplitudes of about one lattice spacing keep every cell well inside the
    # minimum-image range that the GPU path requires
    n, L = 32, 1.0
    y, psi_exact, sdisp = plane_wave(n, L, [0.03, 0.02, 0.04], [0.3, 1.1, -0.4])
    a = L / n
    s = B.Solver(y, [L] * 3, precision="fp64")
    g = s.laguerre(psi_exact)
    np.testing.assert_allclose(g["vol"], a ** 3, rtol=1e-10)
    st = s.solve(1e-10)
    assert st["max_rel_err"] <= 1e-10
    np.testing.assert_allclose(s.displacement(), sdisp, atol=1e-7 * a)


def test_error_codes():
    y, nu, L = c1()
    opt = B.sdot_default_options()
    rc, ctx = B.sdot_create(y, nu * 1.01, [L] * 3, opt)
    assert rc == B.SDOT_ERR_MASS and not ctx
    yd = y.copy()
    yd[5] = yd[9]
    rc, ctx = B.sdot_create(yd, None, [L] * 3, opt)
    assert rc == B.SDOT_ERR_DUPLICATE
    yo = y.copy()
    yo[3, 0] = L
    rc, ctx = B.sdot_create(yo, None, [L] * 3, opt)
    assert rc == B.SDOT_ERR_ARG
    rc, ctx = B.sdot_create(y[:10], None, [L] * 3, opt)
    assert rc == B.SDOT_ERR_TOO_FEW
    # a psi that empties a cell
    s = B.Solver(y, [L] * 3, precision="fp64")
    psi = np.zeros(y.shape[0])
    psi[7] = -50 * (L / 16) ** 2
    g = s.laguerre(psi, allow_empty=True)
    assert g["rc"] == B.SDOT_ERR_EMPTY_CELL and g["vol"][7] == 0.0
    assert abs(g["vol"].sum() - L ** 3) < 1e-10


def test_device_pointers_and_stream():
    y, nu, L = c1()
    pos = torch.from_numpy(y).cuda()
    stream = torch.cuda.Stream()
    rc, ctx = B.sdot_create(pos, torch.from_numpy(nu).cuda(), [L] * 3,
                            B.sdot_default_options(precision="fp64"))
    B.check(rc)
    try:
        B.check(B.sdot_set_stream(ctx, stream))
        vol = torch.empty(y.shape[0], dtype=torch.float64, device="cuda")
        B.check(B.sdot_laguerre(ctx, None, vol, None, None))
        o = O.laguerre(y, np.zeros(y.shape[0]), L, nu, with_hessian=False)
        np.testing.assert_allclose(vol.cpu().numpy(), o["vol"], rtol=1e-10)
    finally:
        B.sdot_destroy(ctx)


def test_c2_sampled_cells_fp64():
    # full 128^3 box of the BBKS spectrum at psi = 0; 40 sampled cells vs the oracle
    y, nu, L = ics.make_config(**ics.CONFIGS["zeldovich-128^3-bbks-1.5a"])
    N = y.shape[0]
    a = L / 128
    s = B.Solver(y, [L] * 3, precision="fp64")
    g = s.laguerre()
    idx = np.random.default_rng(0).choice(N, 40, replace=False)
    o = O.cells(y, np.zeros(N), L, "certified", idx=idx)
    np.testing.assert_allclose(g["vol"][idx], o["vol"], rtol=0, atol=1e-10 * a ** 3)
    assert abs(g["vol"].sum() - L ** 3) < 1e-9 * L ** 3


def _pick(rng, idx, m):
    idx = np.asarray(idx)
    return rng.choice(idx, min(m, idx.size), replace=False) if idx.size else idx


def test_c3_converged_status_selected_cells():
    # The box bench.py times (256^3 lattice + 838 860 points in 2000 clumps of width
    # 0.05a, 17.6 M seeds), solved in mixed precision to max|V - nu|/nu <= 1e-4 in the
    # default launch configuration. At the solution the clump cells have grown and the
    # lattice cells around the clumps sit 2-4 a from their seeds. Cells chosen by what
    # happened to them in the evaluation at the solution (re-queued by the security
    # test, re-clipped in FP64), clump cells and the lattice cells farthest from their
    # seeds are compared with the certified oracle at the same psi; then the same psi is
    # evaluated in FP64 by a fresh context (its first diagram re-queues every cell whose
    # k nearest seeds do not certify it) and compared at 1e-10.
    y, nu, L = ics.make_config(**ics.CONFIGS["zeldovich-256^3-kinv-0.3a+clumps"])
    N = y.shape[0]
    n_lat = 256 ** 3
    a = L / 256
    rng = np.random.default_rng(17)
    pos = torch.from_numpy(y).cuda()
    with B.Solver(pos, [L] * 3, precision="mixed") as s:
        st = s.solve(1e-4)
        assert st["max_rel_err"] <= 1e-4
        psi = s.psi()
        g = s.laguerre(psi)
        status = s.status()
        disp = s.displacement()
    far = np.argsort(-np.linalg.norm(disp[:n_lat], axis=1))[:8]
    assert np.linalg.norm(disp[far[-1]]) >= 1.0 * a
    idx = np.unique(np.concatenate([
        _pick(rng, np.flatnonzero(status & 8), 8),
        _pick(rng, np.flatnonzero(status & (4 | 32 | 64 | 128)), 4),
        n_lat + rng.choice(N - n_lat, 8, replace=False), far]))
    assert idx.size >= 24
    o = O.cells(y, psi, L, "certified", idx=idx)
    cen_o = y[idx] + o["m1"] / o["vol"][:, None]
    ev = np.abs(g["vol"][idx] - o["vol"]) / nu[idx]
    dc = g["centroid"][idx] - cen_o
    dc -= L * np.round(dc / L)
    dd = disp[idx] - (-o["m1"] / o["vol"][:, None])
    print(f"C3 mixed at the solution: {idx.size} cells, max volume error {ev.max():.2e} nu, "
          f"centroid {np.abs(dc).max() / a:.2e} a, displacement {np.abs(dd).max() / a:.2e} a")
    # FP32 cells next to the clumps carry the largest rounding (facet planes of clump
    # seeds nearly parallel, the steepest ones re-clipped in FP64): over all 17.6 M cells
    # of this box the FP32 volume error is at most 1.5e-5 nu, the centroid error 5.4e-6 a
    assert ev.max() <= 3e-5
    assert np.abs(dc).max() <= 2e-5 * a
    assert np.abs(dd).max() <= 2e-5 * a
    with B.Solver(pos, [L] * 3, precision="fp64") as s64:
        g64 = s64.laguerre(psi)
        st64 = s64.status()
    idx64 = np.unique(np.concatenate([idx, _pick(rng, np.flatnonzero(st64 & 8), 8)]))
    o64 = O.cells(y, psi, L, "certified", idx=idx64)
    cen64 = y[idx64] + o64["m1"] / o64["vol"][:, None]
    ev64 = np.abs(g64["vol"][idx64] - o64["vol"]) / o64["vol"]
    dc64 = g64["centroid"][idx64] - cen64
    dc64 -= L * np.round(dc64 / L)
    print(f"C3 FP64 at the same psi: {idx64.size} cells ({int((st64[idx64] & 8).astype(bool).sum())} "
          f"re-queued), max volume error {ev64.max():.2e} rel, centroid "
          f"{np.abs(dc64).max() / a:.2e} a")
    assert ev64.max() <= 1e-10
    assert np.abs(dc64).max() <= 1e-10 * a


def test_solve_fp64_nonuniform_masses():
    # per-seed masses (+-30%), normalised to the box volume: the masses enter through
    # sdot_create in the caller's order
    y, _, L = c1()
    a = L / 16
    N = y.shape[0]
    w = 1.0 + 0.3 * np.random.default_rng(21).uniform(-1.0, 1.0, N)
    nu = w / w.sum() * L ** 3
    s = B.Solver(y, [L] * 3, mass=nu, precision="fp64")
    st = s.solve(1e-10)
    assert st["max_rel_err"] <= 1e-10
    _, info = O.solve(y, nu, L, tol=1e-11)
    assert np.max(np.abs(s.displacement() - info["disp"])) <= 1e-6 * a
    g = s.laguerre(s.psi())
    np.testing.assert_allclose(g["vol"], nu, rtol=1e-9)


def test_fault_paths():
    # non-finite psi is refused without touching the context; the Newton cap reports
    y, nu, L = c1()
    N = y.shape[0]
    s = B.Solver(y, [L] * 3, precision="fp64")
    bad = np.zeros(N)
    bad[17] = np.nan
    assert B.sdot_laguerre(s.ctx, bad, np.empty(N)) == B.SDOT_ERR_ARG
    assert "non-finite" in B.sdot_last_error()
    bad[17] = np.inf
    assert B.sdot_solve(s.ctx, 1e-4, bad) == B.SDOT_ERR_ARG
    st = s.solve(1e-8)
    assert st["max_rel_err"] <= 1e-8
    s.close()
    s2 = B.Solver(y, [L] * 3, precision="fp64", newton_maxit=1)
    assert B.sdot_solve(s2.ctx, 1e-12) == B.SDOT_ERR_MAXIT
    s2.close()
