"""sdot_knn_static: the kNN build for callers that cannot allocate device memory.

Such callers (code inside another framework's memory pool or under a fixed memory
budget, or latency-critical code that must not call cudaMalloc/cudaFree) get the same
neighbour lists as sdot_knn from one fixed scratch array inside the library. Checked
here against the allocating entry point and against the oracle's brute-force lists on
two calls in a row (different boxes, so the second call must not see the first call's
leftovers). This file is collected last.
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


def _inputs():
    y1, _, L1 = ics.make_config(**ics.CONFIGS["zeldovich-16^3-kinv-0.3a"])
    rng = np.random.default_rng(11)
    n = 29
    y2 = np.mod(ics.lattice(n, 2.5) + rng.uniform(-0.3, 0.3, (n ** 3, 3)) * (2.5 / n), 2.5)
    return [(y1, L1, 24), (y2, 2.5, 17)]


def test_knn_static_matches_sdot_knn_twice():
    for y, L, k in _inputs():
        ref = B.Solver(y, [L] * 3, precision="fp64", k=k).knn()
        pos = torch.from_numpy(np.ascontiguousarray(y)).cuda()
        out = torch.full((y.shape[0], k), -7, dtype=torch.int32, device="cuda")
        B.check(B.sdot_knn_static(pos, [L] * 3, k, out))
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
        brute, _ = O.knn(np.ascontiguousarray(y), L, k)
        np.testing.assert_array_equal(out.cpu().numpy(), brute)


def test_knn_static_rejects_oversize():
    n = B.SDOT_STATIC_MAX_N + 1
    pos = torch.rand((n, 3), dtype=torch.float64, device="cuda")
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    assert B.sdot_knn_static(pos, [1.0] * 3, 4, out) == B.SDOT_ERR_ARG
    assert "<=" in B.sdot_last_error()


def test_knn_static_names_itself_in_errors():
    y, _, L = ics.make_config(**ics.CONFIGS["zeldovich-16^3-kinv-0.3a"])
    y = y.copy()
    y[5, 1] = L  # outside [0, L)
    pos = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    out = torch.empty((y.shape[0], 8), dtype=torch.int32, device="cuda")
    assert B.sdot_knn_static(pos, [L] * 3, 8, out) == B.SDOT_ERR_ARG
    assert B.sdot_last_error().startswith("sdot_knn_static:"), B.sdot_last_error()
