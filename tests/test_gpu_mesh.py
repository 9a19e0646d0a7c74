"""phi_I on a mesh, the Zel'dovich move and the Eulerian deposit on the GPU (sdot_mesh,
through the C ABI) against the oracle.

Tolerances: phi_I and the owners are computed by both sides with the same correctly
rounded operations at the same psi, so they agree bitwise; the deposited density is an
exact polyhedral intersection on both sides (FP64 cells, different clipping orders, the
GPU summing in 64-bit fixed point with unit 2^-62 of the box's mass), held to 1e-9
relative.
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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mesh_matches_oracle_at_the_solution(prec):
    y, nu, L = ics.make_config(**ics.CONFIGS["zeldovich-16^3-kinv-0.3a"])
    with B.Solver(y, [L] * 3, precision=prec) as s:
        s.solve(1e-10)
        psi = s.psi()
        out = {(lam, M): s.mesh(lam, M) for lam, M in ((0.0, 16), (0.3, 21), (0.8, 11))}
    for (lam, M), g in out.items():
        rho = O.deposit(y, psi, L, M, lam)
        np.testing.assert_allclose(g["rho"], rho, rtol=1e-9, atol=1e-12)
        assert abs(g["rho"].mean() - 1.0) < 1e-11
        phi, owner = O.potential_mesh(y, psi, L, M)
        np.testing.assert_array_equal(g["phi"], phi)
        np.testing.assert_array_equal(g["owner"], owner)


def test_mesh_plane_wave_closed_form():
    # the cells of the separable plane wave are the lattice cubes: the deposit is a
    # product of 1-D overlaps and the owner of a point is its cube (n = 7, M = 13: no
    # mesh point (m + 1/2)/13 lies on a cube face i/7)
    from test_oracle_pins import _overlap_1d, plane_wave

    n, L, lam, M = 7, 1.0, 0.4, 13
    a = L / n
    amps, phases = [0.03, 0.02, 0.035], [0.3, 1.1, -0.4]
    y, psi, s = plane_wave(n, L, amps, phases)
    with B.Solver(y, [L] * 3, precision="fp64") as sv:
        sv.laguerre(psi)
        g = sv.mesh(lam, M)
    gl = (np.arange(n) + 0.5) * a
    ov = [_overlap_1d(gl + lam * A * np.sin(2 * np.pi * gl / L + ph), (1 - lam) * a, M, L)
          .sum(axis=0) for A, ph in zip(amps, phases)]
    expect = a ** 3 / (L / M) ** 3 * ov[2][:, None, None] * ov[1][None, :, None] * \
        ov[0][None, None, :]
    np.testing.assert_allclose(g["rho"], expect, rtol=1e-9, atol=1e-12)
    gm = (np.arange(M) + 0.5) * L / M
    c = np.floor(gm / a).astype(int)
    np.testing.assert_array_equal(g["owner"], c[None, None, :] + n * c[None, :, None]
                                  + n * n * c[:, None, None])


def test_mesh_argument_errors():
    y, nu, L = ics.make_config(**ics.CONFIGS["zeldovich-16^3-kinv-0.3a"])
    with B.Solver(y, [L] * 3, precision="fp64") as s:
        out = np.empty(8)
        assert B.sdot_mesh(s.ctx, 1.0, 2, out) == B.SDOT_ERR_ARG
        assert B.sdot_mesh(s.ctx, -0.1, 2, out) == B.SDOT_ERR_ARG
        assert B.sdot_mesh(s.ctx, 0.1, 0, out) == B.SDOT_ERR_ARG
        assert B.sdot_mesh(s.ctx, 0.1, 2) == B.SDOT_ERR_ARG
