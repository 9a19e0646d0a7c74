"""The caller's device allocator (sdot_set_allocator) on the GPU: a context whose
memory comes from PyTorch's caching allocator gives the same solve as one on
cudaMalloc, and returns every block it took."""
import numpy as np
import pytest

from paper_2110_08868_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2110_08868_gb300 import binding as B  # noqa: E402


def _solve(y, L):
    s = B.Solver(y, [L] * 3, precision="fp64")
    try:
        st = s.solve(1e-10)
        return st, s.displacement(), s.psi()
    finally:
        s.close()


def test_solve_on_the_torch_pool():
    y, _, L = ics.make_config(**ics.CONFIGS["zeldovich-16^3-kinv-0.3a"])
    ref = _solve(y, L)
    live = {}

    def alloc(n):
        p = torch.cuda.caching_allocator_alloc(n)
        live[p] = n
        return p

    def free(p):
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    B.check(B.sdot_set_allocator(alloc, free))
    try:
        got = _solve(y, L)
    finally:
        B.check(B.sdot_set_allocator())
    assert not live  # every block went back to the pool
    assert got[0]["newton_iters"] == ref[0]["newton_iters"]
    np.testing.assert_array_equal(got[1], ref[1])
    np.testing.assert_array_equal(got[2], ref[2])
