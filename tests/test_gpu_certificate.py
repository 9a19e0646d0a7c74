"""Carried security certificates (the first pass reuses a cell's previous security walk
when psi moved less than the reserves; the certificate's recorded seeds are re-tested
exactly). Whatever the first pass took, the diagram must be the oracle's: a seed the
carried certificate failed to exclude would show as a wrong volume or centroid.

Tolerances as in test_gpu_parity: FP64 1e-10 relative to a^3 and a; mixed 2e-5.
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


def _last(s):
    ei = B.sdot_eval_info()
    B.check(B.sdot_last_eval(s.ctx, ei))
    return ei.as_dict()


def _check(s, y, psi, L, nu, vtol, ctol):
    a = L / round(len(y) ** (1 / 3))
    g = s.laguerre(psi, allow_empty=True)
    info = _last(s)
    o = O.laguerre(y, psi, L, nu)
    np.testing.assert_allclose(g["vol"], o["vol"], rtol=0, atol=vtol * a ** 3)
    ok = o["vol"] > 0
    dc = g["centroid"][ok] - o["centroid"][ok]
    dc -= L * np.round(dc / L)
    assert np.max(np.abs(dc)) <= ctol * a
    return info


@pytest.mark.parametrize("prec,vtol,ctol", [("fp64", 1e-10, 1e-10), ("mixed", 2e-5, 2e-5)])
def test_carried_certificates_match_the_oracle(prec, vtol, ctol):
    y, nu, L = ics.make_config(**ics.CONFIGS["zeldovich-16^3-kinv-0.3a"])
    N = y.shape[0]
    a = L / 16
    s = B.Solver(y, [L] * 3, precision=prec)
    s.solve(1e-6)
    psi = s.psi()
    _check(s, y, psi, L, nu, vtol, ctol)  # records the certificates at the solution
    # within the reserves: psi_j - psi_i moves by at most 0.002 a^2
    rng = np.random.default_rng(11)
    p = psi + 0.001 * a * a * rng.uniform(-1.0, 1.0, N)
    info = _check(s, y, p, L, nu, vtol, ctol)
    assert info["carried"] >= N // 2, info
    # the same psi again: nothing consumed, the carried certificates hold again
    info = _check(s, y, p, L, nu, vtol, ctol)
    assert info["carried"] >= N // 2, info
    # far beyond the reserves: every cell walks again
    q = p.copy()
    q[rng.choice(N, 7, replace=False)] += 0.5 * a * a
    info = _check(s, y, q, L, nu, vtol, ctol)
    assert info["carried"] == 0, info
    # and certificates recorded after that walk carry the next evaluation at q
    info = _check(s, y, q, L, nu, vtol, ctol)
    assert info["carried"] >= N // 2, info


def test_carried_certificates_on_a_clumpy_box_follow_the_solve():
    # a clumpy box through the whole mixed solve: every evaluation near convergence may
    # carry certificates, and the converged diagram must still be the oracle's
    y, _, _ = ics.zeldovich_box(12, 1.0, ics.spectrum_kinv, 0.3, 5)
    y = ics.add_clumps(y, 1.0, 12, 2, 60, 0.05, 7)
    y = np.ascontiguousarray(y)
    N = y.shape[0]
    nu = np.full(N, 1.0 / N)
    s = B.Solver(y, [1.0] * 3, precision="mixed")
    st = s.solve(1e-5)
    assert st["max_rel_err"] <= 1e-5
    psi = s.psi()
    _check(s, y, psi, 1.0, nu, 2e-5, 2e-5)
    info = _check(s, y, psi, 1.0, nu, 2e-5, 2e-5)
    assert info["carried"] > 0, info
    # cells next to the clumps fail the FP32 check and are re-clipped in FP64, where the
    # certificate the first pass kept for them replaces the walk as well
    print("clumpy box: %d cells carried, %d re-clipped in FP64" %
          (info["carried"], info["reclipped_fp64"]))
