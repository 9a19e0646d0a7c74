"""Mixed precision against FP64 on a clumpy box (the regime of the 256^3 + clumps
workload, small enough for a test).

The box is a 20^3 Zel'dovich lattice plus two Gaussian clumps of 420 points of width
0.05 lattice spacings. It is solved in FP64, then the diagram at the solution is
evaluated with FP32 cells. The clump seeds are 0.05 spacings apart, and the lattice
cells around a clump end up 2-4 spacings from their own seeds, bounded by the
nearly parallel bisectors of the clump seeds: the hardest case for FP32 geometry.
FP32 polytopes are held relative to a frame at the cell's previous centroid (a cell
of a fresh context is clipped again in a frame at its first centroid), which removes
the part of the rounding that grows with the distance between a cell and its seed.
The bound below is the measured FP32 error of this case with a safety factor; the
mixed solver only relies on FP32 until its line search stalls, then finishes in FP64.
"""
import numpy as np
import pytest

from paper_2110_08868_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2110_08868_gb300 import binding as B  # noqa: E402


def clumpy_box():
    n, L = 20, 1.0
    y, _, _ = ics.zeldovich_box(n, L, ics.spectrum_kinv, 0.3, 7)
    y = ics.add_clumps(y, L, n, 2, 840, 0.05, 8)
    return np.ascontiguousarray(y), ics.uniform_masses(y.shape[0], L), L


def test_mixed_vs_fp64_on_clumps():
    y, nu, L = clumpy_box()
    s64 = B.Solver(y, [L] * 3, precision="fp64")
    st = s64.solve(1e-9)
    assert st["max_rel_err"] <= 1e-9
    psi = s64.psi()
    g64 = s64.laguerre(psi)
    s32 = B.Solver(y, [L] * 3, precision="mixed")
    # a fresh context (cells re-clipped in frames at their first centroids), then a
    # warm one (frames at the previous centroids); measured max 4.4e-6 for both
    for _ in range(2):
        g32 = s32.laguerre(psi)
        err = np.abs(g32["vol"] - g64["vol"]) / nu
        assert abs(g32["vol"].sum() - L ** 3) < 1e-6 * L ** 3
        assert err.max() < 2e-5, (err.max(), int(err.argmax()))
    # the mixed solver itself reaches the criterion (FP64 refinement if needed)
    st32 = s32.solve(1e-6)
    assert st32["max_rel_err"] <= 1e-6
