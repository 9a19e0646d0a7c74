"""Argument validation of the C ABI (include/sdot.h), on the host: every check below
returns before the library touches the device, so it runs without a GPU. The codes are
the ones the header documents for each call."""
import ctypes

import numpy as np
import pytest

from paper_2110_08868_gb300 import binding as B
from paper_2110_08868_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    B.load()


def _pos(n, seed=0):
    return np.random.default_rng(seed).uniform(0.0, 1.0, (n, 3))


def test_default_options():
    o = B.sdot_default_options()
    assert (o.k, o.precision, o.seeds_per_leaf, o.cg_rtol) == (24, B.SDOT_PREC_MIXED, 2.0, 1e-3)
    assert (o.cg_maxit, o.newton_maxit, o.warm_alpha, o.verbose) == (5000, 100, 1, 0)
    assert o.carry_certificates == 1
    assert o.alpha_min == 2.0 ** -30
    so = B.sdot_server_default_options()
    assert (so.hbm_budget, so.max_active, so.device, so.batch_clip) == (0, 8, -1, 1)


@pytest.mark.parametrize("n", [0, 1])
def test_create_needs_two_seeds(n):
    rc, ctx = B.sdot_create(_pos(max(n, 1))[:n], None, [1.0] * 3)
    assert rc == B.SDOT_ERR_ARG and not ctx.value
    assert "2 <= N" in B.sdot_last_error()


@pytest.mark.parametrize("box", [[1.0, 0.0, 1.0], [1.0, -2.0, 1.0], [np.inf, 1.0, 1.0],
                                 [np.nan, 1.0, 1.0]])
def test_create_rejects_bad_boxes(box):
    rc, ctx = B.sdot_create(_pos(100), None, box)
    assert rc == B.SDOT_ERR_ARG and not ctx.value


@pytest.mark.parametrize("kw", [dict(k=0), dict(k=65), dict(precision=2),
                                dict(seeds_per_leaf=0.0), dict(cg_rtol=0.0), dict(cg_rtol=1.0),
                                dict(cg_maxit=0), dict(newton_maxit=-1), dict(alpha_min=0.0),
                                dict(alpha_min=2.0), dict(carry_certificates=2),
                                dict(carry_certificates=-1)])
def test_create_rejects_bad_options(kw):
    rc, ctx = B.sdot_create(_pos(100), None, [1.0] * 3, B.sdot_default_options(**kw))
    assert rc == B.SDOT_ERR_ARG and not ctx.value
    assert "invalid options" in B.sdot_last_error()


def test_create_k_needs_enough_seeds():
    rc, ctx = B.sdot_create(_pos(20), None, [1.0] * 3, B.sdot_default_options(k=24))
    assert rc == B.SDOT_ERR_TOO_FEW and not ctx.value


def test_null_context_calls():
    lib = B.load()
    null = ctypes.c_void_p()
    assert B.sdot_solve(null, 1e-4) == B.SDOT_ERR_ARG
    assert B.sdot_laguerre(null) == B.SDOT_ERR_ARG
    assert B.sdot_get_psi(null, np.empty(4)) == B.SDOT_ERR_ARG
    assert B.sdot_displacement(null, np.empty((4, 3))) == B.SDOT_ERR_ARG
    assert B.sdot_size(null)[0] == B.SDOT_ERR_ARG
    assert lib.sdot_set_stream(null, None) == B.SDOT_ERR_ARG
    assert lib.sdot_knn(null, None) == B.SDOT_ERR_ARG
    assert lib.sdot_cell_status(null, None) == B.SDOT_ERR_ARG
    assert lib.sdot_csr_copy(None, None, None, None) == B.SDOT_ERR_ARG
    assert lib.sdot_default_options(None) == B.SDOT_ERR_ARG
    B.sdot_destroy(null)  # NULL is accepted


def test_knn_static_limits():
    lib = B.load()
    b = np.ones(3)
    bp = ctypes.c_void_p(b.ctypes.data)
    fake = ctypes.c_void_p(16)  # never dereferenced: the size checks come first
    assert lib.sdot_knn_static(fake, B.SDOT_STATIC_MAX_N + 1, bp, 24, fake, None) == B.SDOT_ERR_ARG
    assert lib.sdot_knn_static(fake, 1000, bp, B.SDOT_STATIC_MAX_K + 1, fake, None) == B.SDOT_ERR_ARG
    assert lib.sdot_knn_static(fake, 1, bp, 1, fake, None) == B.SDOT_ERR_ARG
    assert lib.sdot_knn_static(fake, 10, bp, 10, fake, None) == B.SDOT_ERR_ARG  # k >= N
    assert lib.sdot_knn_static(None, 10, bp, 3, fake, None) == B.SDOT_ERR_ARG


def test_server_null_and_argument_errors():
    lib = B.load()
    null = ctypes.c_void_p()
    st = ctypes.c_int()
    jid = ctypes.c_int64()
    assert lib.sdot_server_poll(null, 1, ctypes.byref(st)) == B.SDOT_ERR_ARG
    assert lib.sdot_server_wait(null, 1, 0.0, ctypes.byref(st)) == B.SDOT_ERR_ARG
    assert lib.sdot_server_result(null, 1, None, None, None, None) == B.SDOT_ERR_ARG
    assert lib.sdot_server_get_info(null, None) == B.SDOT_ERR_ARG
    b = np.ones(3)
    p = _pos(100)
    assert lib.sdot_server_submit(null, ctypes.c_void_p(p.ctypes.data), None, 100,
                                  ctypes.c_void_p(b.ctypes.data), None, 1e-4,
                                  ctypes.byref(jid)) == B.SDOT_ERR_ARG
    assert lib.sdot_server_create(None, None) == B.SDOT_ERR_ARG
    B.sdot_server_destroy(null)  # NULL is accepted


def test_error_codes_are_distinct_and_named():
    codes = [v for v in B.ERRORS]
    assert len(set(codes)) == len(codes) == 12
    assert sorted(codes) == list(range(-12, 0))


def test_injected_allocator_failure_reports_oom():
    # the caller's allocator refuses the first request: sdot_create stops there, frees
    # nothing it did not get, and reports SDOT_ERR_OOM
    calls = []

    def alloc(n):
        calls.append(n)
        return 0

    def free(p):
        raise AssertionError("nothing was allocated")

    assert B.sdot_set_allocator(alloc, free) == B.SDOT_OK
    try:
        rc, ctx = B.sdot_create(_pos(1000), None, [1.0] * 3)
        assert rc == B.SDOT_ERR_OOM and not ctx.value
        assert len(calls) == 1
        assert "caller's allocator" in B.sdot_last_error()
    finally:
        assert B.sdot_set_allocator() == B.SDOT_OK


def test_injected_allocator_partial_failure_frees_through_it():
    # the allocator hands out 5 (never dereferenced) addresses, then fails: every
    # address it gave is returned to it exactly once, none to cudaFree
    given, freed = [], []

    def alloc(n):
        if len(given) == 5:
            return 0
        given.append(0x10000000 * (len(given) + 1))
        return given[-1]

    assert B.sdot_set_allocator(alloc, freed.append) == B.SDOT_OK
    try:
        rc, ctx = B.sdot_create(_pos(1000), None, [1.0] * 3)
        assert rc == B.SDOT_ERR_OOM and not ctx.value
        assert sorted(freed) == sorted(given) and len(given) == 5
    finally:
        assert B.sdot_set_allocator() == B.SDOT_OK


def test_allocator_needs_both_functions():
    assert B.sdot_set_allocator(alloc=lambda n: 0) == B.SDOT_ERR_ARG
    assert B.sdot_set_allocator(free=lambda p: None) == B.SDOT_ERR_ARG
    assert B.sdot_set_allocator() == B.SDOT_OK


def test_wrappers_are_context_managers():
    assert hasattr(B.Solver, "__enter__") and hasattr(B.Solver, "__exit__")
    assert hasattr(B.Server, "__enter__") and hasattr(B.Server, "__exit__")


class _FakeCudaTensor:
    """Just enough of a CUDA tensor for the binding's shape checks (no device needed)."""

    def __init__(self, shape, device="cuda:0"):
        self.shape = tuple(shape)
        self.is_cuda = True
        self.device = device

    def dim(self):
        return len(self.shape)


@pytest.mark.parametrize("pos_shape,nbr_shape,k,devs,msg", [
    ((100, 2), (100, 8), 8, ("cuda:0", "cuda:0"), "pos must have shape (N, 3)"),
    ((100, 3, 1), (100, 8), 8, ("cuda:0", "cuda:0"), "pos must have shape (N, 3)"),
    ((100, 3), (100, 7), 8, ("cuda:0", "cuda:0"), "nbr must have shape (100, 8)"),
    ((100, 3), (99, 8), 8, ("cuda:0", "cuda:0"), "nbr must have shape (100, 8)"),
    ((100, 3), (100 * 8,), 8, ("cuda:0", "cuda:0"), "nbr must have shape (100, 8)"),
    ((100, 3), (100, 8), 8, ("cuda:0", "cuda:1"), "same device"),
])
def test_knn_static_wrapper_rejects_bad_buffers(pos_shape, nbr_shape, k, devs, msg):
    # the C call cannot see buffer sizes, so the binding refuses them before calling it
    pos = _FakeCudaTensor(pos_shape, devs[0])
    nbr = _FakeCudaTensor(nbr_shape, devs[1])
    with pytest.raises(ValueError, match=msg.replace("(", r"\(").replace(")", r"\)")):
        B.sdot_knn_static(pos, [1.0] * 3, k, nbr)


def test_knn_static_wrapper_rejects_host_buffers():
    with pytest.raises(ValueError, match="CUDA tensor"):
        B.sdot_knn_static(_pos(100), [1.0] * 3, 8, np.zeros((100, 8), np.int32))


def test_power_spectrum_argument_checks_need_no_gpu():
    # sdot_power_spectrum refuses bad arguments before touching the device
    rho = np.ones((8, 8, 8))
    for L, nbins in ((0.0, 4), (-1.0, 4), (np.inf, 4), (np.nan, 4), (1.0, 0), (1.0, 17)):
        with pytest.raises(B.SdotError) as e:
            B.sdot_power_spectrum(rho, L, nbins)
        assert e.value.code == B.SDOT_ERR_ARG
        assert "sdot_power_spectrum" in B.sdot_last_error()
    with pytest.raises(B.SdotError):
        B.sdot_power_spectrum(np.ones((1, 1, 1)), 1.0, 1)  # M < 2
    with pytest.raises(ValueError):
        B.sdot_power_spectrum(np.ones((8, 8, 4)), 1.0, 4)  # not a cube
