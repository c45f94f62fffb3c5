"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the solver: it only draws permeability
fields and lists the workload parameters.  Both sides consume the exact same
bytes it returns.

Permeability: the paper's model problem (Sec. 5) uses a constant K.  The
larger workloads use a log-normal field, ln K ~ N(mean, sigma^2), with the
isotropic exponential covariance C(r) = sigma^2 exp(-r / ell), r and ell in
cell units, sampled on the n x n Darcy grid by circulant embedding on a
periodic M x M torus (M >= max(2n, n + 8 ell), a power of two) with numpy's
FFT and PCG64 generator.  Negative embedding eigenvalues are clipped to zero
and their share of the spectrum is reported.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def constant_K(n: int, value: float = 1.0) -> np.ndarray:
    return np.full((n, n), float(value))


def lognormal_K(n: int, mean: float = -4.0, sigma: float = 1.0, corr_len: float = 16.0,
                seed: int = 0, return_info: bool = False):
    """Log-normal permeability on the n x n pm cells, indexed [j, i] (j = 0 at y = 0)."""
    m = 1
    while m < max(2 * n, n + int(math.ceil(8 * corr_len))):
        m *= 2
    a = np.minimum(np.arange(m), m - np.arange(m)).astype(np.float64)
    r = np.sqrt(a[:, None] ** 2 + a[None, :] ** 2)
    c = sigma * sigma * np.exp(-r / corr_len)
    lam = np.fft.fft2(c).real
    neg = float(-lam[lam < 0].sum() / np.abs(lam).sum()) if np.any(lam < 0) else 0.0
    lam = np.clip(lam, 0.0, None)
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    g = np.fft.fft2(np.sqrt(lam / (m * m)) * eps).real[:n, :n]
    K = np.exp(mean + g)
    if return_info:
        return K, {"embed": m, "clipped_fraction": neg}
    return K


@dataclass
class Workload:
    """One synthetic run: grid, physics, step count and solver precision."""
    name: str
    n: int
    mu: float
    alpha: float
    dt: float
    steps: int
    precision: str          # "fp64" or "mixed"
    K_kind: str = "const"   # "const" or "lognormal"
    K_mean: float = -4.0
    K_sigma: float = 1.0
    K_seed: int = 0
    K_const: float = 1.0
    extra: dict = field(default_factory=dict)

    def K(self) -> np.ndarray:
        if self.K_kind == "const":
            return constant_K(self.n, self.K_const)
        return lognormal_K(self.n, self.K_mean, self.K_sigma, 16.0, self.K_seed)

    @property
    def dof(self) -> int:
        return 4 * self.n * self.n + 2 * self.n


def mms_small(n: int = 32) -> Workload:
    """Manufactured-solution case: unit coefficients, 10 steps of dt = 0.1."""
    return Workload("mms", n, 1.0, 1.0, 0.1, 10, "fp64")


def lognormal_at_scale(n: int = 1024, precision: str = "fp64", steps: int = 20) -> Workload:
    """mu = 1e-3, ln K ~ N(-4, 1) with correlation length 16 cells, alpha = 1, dt = 0.05."""
    return Workload("lognormal", n, 1e-3, 1.0, 0.05, steps, precision, "lognormal", -4.0, 1.0, 0)


def batch_instances(count: int = 256, seed: int = 0, sizes=(64, 128, 256, 512), steps: int = 10):
    """Independent instances with uneven grids, sigma_lnK in [0.5, 2], alpha log-uniform in [0.1, 10]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        n = int(rng.choice(sizes))
        sig = float(rng.uniform(0.5, 2.0))
        alpha = float(10 ** rng.uniform(-1.0, 1.0))
        out.append(Workload("batch%d" % k, n, 1e-3, alpha, 0.1, steps, "mixed", "lognormal", -4.0, sig,
                            int(rng.integers(0, 2**31 - 1))))
    return out


def serving_requests(count: int, rate: float, seed: int = 0, n_min: int = 32, n_max: int = 1024):
    """Poisson arrivals (rate per second) of runs with log-uniform grids and 5-50 steps.

    A log-uniform draw in [n_min, n_max) is rounded to the nearest m * 2^k with
    m in 4..8 and 2^k <= draw / 4, so that every hierarchy halves down to an
    m x m grid of at most 8 x 8 cells (n = 40, 48, 56, ..., 896, 1024).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        n_raw = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        kexp = max(0, int(math.floor(math.log2(n_raw / 4.0))))
        m = max(4, min(8, int(round(n_raw / 2 ** kexp))))
        n = m * 2 ** kexp
        steps = int(rng.integers(5, 51))
        wl = Workload("req%d" % k, n, 1e-3, 1.0, 0.1, steps, "mixed", "lognormal", -4.0, 1.0,
                      int(rng.integers(0, 2**31 - 1)))
        reqs.append((t, wl))
    return reqs
