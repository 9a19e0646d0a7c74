"""Power spectrum of a density mesh (sdot_power_spectrum) and the fractional BAO signal
d(k) = P_wig(k) / P_nw(k) - 1 of a synthetic wiggle / no-wiggle pair (Sec. "BAO
reconstruction", Fig. 2), against the oracle.

Tolerances: the GPU sums each bin in 64-bit fixed point (unit 2^-38 of the bin's largest
|delta_k|^2), so P agrees with the oracle's FP64 sums to ~1e-10 relative; mode counts are
exact. The end-to-end d(k) compares two solves that stop at different tolerances
(GPU 1e-9, oracle 1e-10 of the volumes), so the densities differ by ~1e-9 relative.
"""
import time

import numpy as np
import pytest

import sdot_oracle as O
from paper_2110_08868_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2110_08868_gb300 import binding as B  # noqa: E402


def test_power_spectrum_matches_the_oracle():
    rng = np.random.default_rng(31)
    M, L = 32, 7.0
    rho = np.exp(0.3 * rng.standard_normal((M, M, M)))
    for nbins in (M // 2, 2 * M):
        P, k, n = B.sdot_power_spectrum(rho, L, nbins)
        Po, ko, no = O.power_spectrum(rho, L, nbins)
        np.testing.assert_array_equal(n, no)
        np.testing.assert_allclose(P, Po, rtol=1e-9, atol=0)
        np.testing.assert_allclose(k, ko, rtol=1e-9, atol=0)
    # the same mesh from device memory, on a stream: the same bits
    rho_d = torch.from_numpy(rho).cuda()
    st = torch.cuda.Stream()
    P2, k2, n2 = B.sdot_power_spectrum(rho_d, L, 2 * M, stream=st)
    np.testing.assert_array_equal(P2, P)
    np.testing.assert_array_equal(k2, k)


def test_power_spectrum_plane_wave_and_odd_mesh():
    # all the power of A cos(2 pi 3 x / L) in bin 3; an odd mesh has no Nyquist plane
    for M in (16, 15):
        L, A = 5.0, 0.3
        x = (np.arange(M) + 0.5) * L / M
        rho = np.broadcast_to(1.0 + A * np.cos(2 * np.pi * 3 * x / L), (M, M, M)).copy()
        P, _, n = B.sdot_power_spectrum(rho, L)
        Po, _, no = O.power_spectrum(rho, L)
        np.testing.assert_array_equal(n, no)
        assert abs(P[2] - 2 * L ** 3 * (A / 2) ** 2 / n[2]) <= 1e-9 * P[2]
        assert np.all(np.abs(np.delete(P, 2)) <= 1e-20)


def test_power_spectrum_argument_errors():
    rho = np.ones((8, 8, 8))
    for args in ((rho, 0.0, 4), (rho, 1.0, 0), (rho, 1.0, 17), (rho, np.inf, 4)):
        with pytest.raises(B.SdotError):
            B.sdot_power_spectrum(*args)
    with pytest.raises(B.SdotError):
        B.sdot_power_spectrum(np.zeros((8, 8, 8)), 1.0, 4)  # mean 0
    with pytest.raises(ValueError):
        B.sdot_power_spectrum(np.ones((8, 8, 4)), 1.0, 4)


def test_fractional_bao_signal_of_a_wiggle_pair_matches_the_oracle():
    # a wiggle / no-wiggle pair with the same phases (the same seed; the sine term of the
    # spectrum switched off), each solved, its cells moved to lambda and deposited, then
    # d(k) = P_wig / P_nw - 1; the same chain through the oracle
    n, L, M, lam = 16, 1000.0, 16, 0.1  # box in Mpc/h, k in h/Mpc as the BBKS spectrum takes
    d = {}
    for impl in ("gpu", "oracle"):
        P = {}
        for amp in (0.1, 0.0):
            spec = lambda k, amp=amp: ics.spectrum_bbks_wiggle(k, wiggle_amp=amp)  # noqa: E731
            y, _, _ = ics.zeldovich_box(n, L, spec, 0.3, 41)
            y = np.ascontiguousarray(y)
            nu = np.full(n ** 3, L ** 3 / n ** 3)
            if impl == "gpu":
                s = B.Solver(y, [L] * 3, precision="fp64")
                st = s.solve(1e-9)
                assert st["max_rel_err"] <= 1e-9
                rho = s.mesh(lam, M)["rho"]
                P[amp] = B.sdot_power_spectrum(rho, L)[0]
                s.close()
            else:
                psi, info = O.solve(y, nu, L, tol=1e-10)
                rho = O.deposit(y, psi, L, M, lam)
                P[amp] = O.power_spectrum(rho, L)[0]
        d[impl] = P[0.1] / P[0.0] - 1.0
    assert np.all(np.isfinite(d["gpu"]))
    np.testing.assert_allclose(d["gpu"], d["oracle"], rtol=0, atol=1e-6)


def test_power_spectrum_time_512():
    # one estimator call on a 512^3 device mesh (1 GiB), timed for the record
    M = 512
    g = torch.Generator(device="cuda").manual_seed(5)
    rho = torch.rand((M, M, M), dtype=torch.float64, device="cuda", generator=g) + 0.5
    B.sdot_power_spectrum(rho, 1000.0, M // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P, _, n = B.sdot_power_spectrum(rho, 1000.0, M // 2)
    dt = time.perf_counter() - t0
    print(f"power spectrum 512^3: {dt * 1e3:.1f} ms per call (allocation, transform, binning)")
    assert n.sum() > 0 and np.all(P[1:] > 0)
