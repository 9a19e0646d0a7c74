"""Seeded synthetic inputs: Zel'dovich-displaced lattices in a periodic box.

This module produces the point sets (y_j, nu_j) that both the CUDA path and the
CPU oracle consume. It holds none of the transport method's arithmetic: it only
draws a Gaussian random displacement field and moves lattice points by it.

The paper reconstructs FastPM and AbacusCosmos particle snapshots (Sec. "BAO
reconstruction"), which are not available here. These boxes stand in for them:
the final positions are x = q + s(q) with q on a uniform lattice (the uniform
initial density rho_I = 1 of Sec. "Monge-Ampere-Kantorovich Reconstruction")
and s the Zel'dovich displacement of a Gaussian field (the LPT step named at the
end of the same section).

Recipe (every call is deterministic in ``seed``; numpy PCG64):
  white noise n^3 ~ N(0,1) -> rfftn -> multiply by sqrt(P(|k|)) -> zero k = 0 and
  every |k| >= k_Nyquist = pi n / L (spherical cut) -> s_a(k) = i k_a / k^2 delta(k)
  -> irfftn -> scale so that the 3D rms of |s| equals ``rms`` lattice spacings ->
  y = q + s with q = (i + 1/2) a, wrapped into [0, L).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "spectrum_kinv",
    "spectrum_bbks_wiggle",
    "zeldovich_box",
    "add_clumps",
    "uniform_masses",
    "lattice",
    "CONFIGS",
    "make_config",
    "serving_stream",
]


def spectrum_kinv(k):
    """P(k) proportional to 1/k (amplitude irrelevant after rms scaling)."""
    return 1.0 / k


def _bbks_transfer(q):
    # Bardeen, Bond, Kaiser & Szalay (1986) fitting form, q = k / Gamma.
    q = np.maximum(q, 1e-30)
    x = 2.34 * q
    poly = 1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4
    return np.log1p(x) / x * poly ** -0.25


def spectrum_bbks_wiggle(k, gamma=0.21, wiggle_amp=0.1, wiggle_scale=105.0):
    """P(k) = k T_BBKS(k/Gamma)^2 (1 + 0.1 sin(105 k)/(105 k)); k in h/Mpc.

    The sine term is a toy acoustic wiggle at 105 Mpc/h standing in for the BAO
    feature of the paper's wiggle/no-wiggle simulation pairs.
    """
    t = _bbks_transfer(k / gamma)
    kr = wiggle_scale * k
    return k * t * t * (1.0 + wiggle_amp * np.sin(kr) / kr)


def lattice(n, L):
    """Cell-centred lattice q = (i + 1/2) a, shape (n^3, 3), x fastest."""
    a = L / n
    g = (np.arange(n, dtype=np.float64) + 0.5) * a
    qz, qy, qx = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)


def zeldovich_box(n, L, spectrum, rms, seed):
    """Return (y, q, s) for an n^3 lattice displaced by a Gaussian field.

    ``rms`` is the target 3D rms of |s| in units of the lattice spacing a = L/n.
    y is wrapped into [0, L); s is the unwrapped displacement.
    """
    rng = np.random.default_rng(seed)
    a = L / n
    white = rng.standard_normal((n, n, n))
    dk = np.fft.rfftn(white)
    kf = 2.0 * np.pi / L
    k1 = np.fft.fftfreq(n, d=1.0 / n) * kf
    k3 = np.fft.rfftfreq(n, d=1.0 / n) * kf
    kz = k1[:, None, None]
    ky = k1[None, :, None]
    kx = k3[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    knyq = np.pi * n / L
    keep = (kk > 0) & (kk < knyq)
    amp = np.zeros_like(kk)
    amp[keep] = np.sqrt(spectrum(kk[keep]))
    dk = dk * amp
    inv_k2 = np.zeros_like(kk)
    inv_k2[keep] = 1.0 / (kk[keep] ** 2)
    comps = []
    for kc in (kx, ky, kz):
        sk = 1j * kc * inv_k2 * dk
        comps.append(np.fft.irfftn(sk, s=(n, n, n), axes=(0, 1, 2)))
    # array index order is (z, y, x); flatten to match lattice() (x fastest)
    s = np.stack([c.ravel() for c in comps], axis=1)
    cur = np.sqrt(np.mean(np.sum(s * s, axis=1)))
    if cur > 0:
        s *= rms * a / cur
    q = lattice(n, L)
    y = np.mod(q + s, L)
    # np.mod can return L for tiny negative inputs; keep the half-open box
    y[y >= L] -= L
    return y, q, s


def add_clumps(y, L, n_side, n_clumps, n_extra, sigma_spacings, seed):
    """Append ``n_extra`` points in ``n_clumps`` compact Gaussian clumps.

    Clump centres are uniform in the box; clump sizes differ by at most one
    point; each point is N(centre, (sigma a)^2) per axis, wrapped.
    """
    rng = np.random.default_rng(seed)
    a = L / n_side
    centres = rng.uniform(0.0, L, size=(n_clumps, 3))
    base, rem = divmod(n_extra, n_clumps)
    sizes = np.full(n_clumps, base, dtype=np.int64)
    sizes[:rem] += 1
    owner = np.repeat(np.arange(n_clumps), sizes)
    pts = centres[owner] + rng.standard_normal((n_extra, 3)) * (sigma_spacings * a)
    pts = np.mod(pts, L)
    pts[pts >= L] -= L
    return np.concatenate([y, pts], axis=0)


def uniform_masses(N, L):
    """nu_j = |box| / N, so the masses sum to the Lagrangian volume (rho_I = 1)."""
    return np.full(N, (L ** 3) / N, dtype=np.float64)


# The five synthetic workloads: name -> parameters.
CONFIGS = {
    "zeldovich-16^3-kinv-0.3a": dict(n=16, L=1.0, spectrum="kinv", rms=0.3, seed=1),
    "zeldovich-128^3-bbks-1.5a": dict(n=128, L=1000.0, spectrum="bbks", rms=1.5, seed=2),
    "zeldovich-256^3-kinv-0.3a+clumps": dict(
        n=256, L=1.0, spectrum="kinv", rms=0.3, seed=3,
        clumps=dict(n_clumps=2000, n_extra=838860, sigma=0.05)),
    "zeldovich-512^3-kinv-1.5a": dict(n=512, L=2000.0, spectrum="kinv", rms=1.5, seed=5),
}


def make_config(n, L, spectrum, rms, seed, clumps=None):
    """Build (y, nu, L) for a parameter set of the form stored in CONFIGS."""
    spec = {"kinv": spectrum_kinv, "bbks": spectrum_bbks_wiggle}[spectrum]
    y, _, _ = zeldovich_box(n, L, spec, rms, seed)
    if clumps:
        y = add_clumps(y, L, n, clumps["n_clumps"], clumps["n_extra"],
                       clumps["sigma"], seed + 100)
    return np.ascontiguousarray(y), uniform_masses(y.shape[0], L), float(L)


def serving_stream(n_jobs=64, seed=4, lo=32, hi=128):
    """The serving workload: job sizes and Poisson arrival gaps.

    Job j is a periodic unit box of N_j = n_j^3 seeds, n_j = round(exp(U(ln lo, ln hi)))
    (log-uniform in the side, hence in N), displaced by the 1/k spectrum at 0.3 lattice
    spacings rms with seed 1000 + j. Returns (sides, gaps): gaps are the inter-arrival
    times of a unit-rate Poisson process (gaps[0] = 0); divide them by the arrival rate.
    """
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), n_jobs))).astype(int)
    gaps = rng.standard_exponential(n_jobs)
    gaps[0] = 0.0
    return sides, gaps
