"""Seeded synthetic inputs: permeability fields, initial saturations, decompositions.

This module only manufactures inputs. It holds none of the method's arithmetic
(no mobility, no fluxes, no local solves), so both the CUDA path and the CPU
oracle read identical arrays from it and neither depends on the other.

The fields stand in for the paper's permeability data (Section 5: the Gaussian
field of Section 5.1, the SPE10-derived layer of Section 5.2 and the fractured
field of Section 5.3 are not distributed with the paper):

* ``lognormal_grf``: log K is a stationary Gaussian random field sampled on the
  cell centres by circulant embedding of the covariance on a periodic grid of
  twice the size (Dietrich & Newsam, SIAM J. Sci. Comput. 18, 1997); negative
  eigenvalues of the embedding are clipped to zero.  Covariances:
  ``exponential``  C(r) = sigma2 * exp(-r / ell)
  ``gaussian``     C(r) = sigma2 * exp(-(r / ell)^2)
* ``channelised``: binary field with sinusoidal channels along x.
* ``fingering_s0``: the viscous-fingering initial saturation (water-filled strip
  at the inlet plus seeded uniform noise), Section 5.4.

All arrays are float64, C-contiguous, shaped [ny][nx] (row j = y index,
column i = x index), cell (i, j) centred at ((i + 1/2) h, (j + 1/2) h).
"""
from __future__ import annotations

import numpy as np


def lognormal_grf(nx: int, ny: int, h: float, sigma2: float, ell: float,
                  cov: str = "exponential", seed: int = 0,
                  mean_log: float = 0.0) -> np.ndarray:
    """K = exp(mean_log + Y), Y a zero-mean GRF with the named covariance."""
    rng = np.random.default_rng(seed)
    mx, my = 2 * nx, 2 * ny
    dx = np.minimum(np.arange(mx), mx - np.arange(mx)) * h
    dy = np.minimum(np.arange(my), my - np.arange(my)) * h
    r = np.sqrt(dx[None, :] ** 2 + dy[:, None] ** 2)
    if cov == "exponential":
        c = sigma2 * np.exp(-r / ell)
    elif cov == "gaussian":
        c = sigma2 * np.exp(-(r / ell) ** 2)
    else:
        raise ValueError(f"unknown covariance {cov!r}")
    lam = np.fft.fft2(c).real
    lam = np.clip(lam, 0.0, None)
    xi = rng.standard_normal((my, mx)) + 1j * rng.standard_normal((my, mx))
    y = np.fft.fft2(np.sqrt(lam / (mx * my)) * xi)
    field = y.real[:ny, :nx]
    return np.ascontiguousarray(np.exp(mean_log + field))


def channelised(nx: int, ny: int, k_channel: float = 1.0, k_matrix: float = 1e-4,
                coverage: float = 0.30, width_range=(8, 24), seed: int = 3) -> np.ndarray:
    """Binary K with sinusoidal channels y_c(x) = y0 + A sin(2 pi x / L + phi).

    Channels (width drawn uniformly in ``width_range`` cells) are added until
    at least ``coverage`` of the cells carry ``k_channel``.
    """
    rng = np.random.default_rng(seed)
    K = np.full((ny, nx), k_matrix)
    xs = np.arange(nx) + 0.5
    yy = np.arange(ny)[:, None] + 0.5
    for _ in range(10000):
        if np.mean(K == k_channel) >= coverage:
            break
        width = rng.integers(width_range[0], width_range[1] + 1)
        y0 = rng.uniform(0, ny)
        amp = rng.uniform(0.02, 0.12) * ny
        wavelength = rng.uniform(0.3, 1.0) * nx
        phase = rng.uniform(0, 2 * np.pi)
        yc = y0 + amp * np.sin(2 * np.pi * xs / wavelength + phase)
        K[np.abs(yy - yc[None, :]) < width / 2] = k_channel
    return np.ascontiguousarray(K)


def fingering_s0(nx: int, ny: int, inlet_frac: float = 0.05, noise_cols: int = 8,
                 noise_amp: float = 0.01, seed: int = 5) -> np.ndarray:
    """s0 = 1 for x < inlet_frac, noise_amp * U[0,1) in the next columns, else 0."""
    rng = np.random.default_rng(seed)
    s0 = np.zeros((ny, nx))
    n_in = max(1, int(round(inlet_frac * nx)))
    s0[:, :n_in] = 1.0
    s0[:, n_in:n_in + noise_cols] = noise_amp * rng.random((ny, min(noise_cols, nx - n_in)))
    return np.ascontiguousarray(s0)


def uneven_widths(total: int, parts, seed: int) -> list[int]:
    """Seeded permutation of ``parts`` (which must sum to ``total``)."""
    parts = list(parts)
    if sum(parts) != total:
        raise ValueError("parts must sum to total")
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.permutation(parts)]


# Workloads used by the tests and the benchmark: grid, subdomain layout, covariance of the
# log-permeability field, viscosity ratio and rebuild threshold of each, listed per entry.
WORKLOADS = {
    # 64x64, 4x4 subdomains of 16x16, exponential GRF (ell 0.1, var 1), M = 1,
    # rebuild every step (eta < 0).
    "gaussian64": dict(nx=64, ny=64, ncx=4, ncy=4, sigma2=1.0, ell=0.1, cov="exponential",
                       seed=1, M=1.0, eta=-1.0, steps=20),
    # 256x256, 16x16 subdomains, Gaussian covariance (ell 0.05, var 4), M = 5, eta = 0.1.
    "gaussian256": dict(nx=256, ny=256, ncx=16, ncy=16, sigma2=4.0, ell=0.05, cov="gaussian",
                        seed=2, M=5.0, eta=0.1, steps=500),
}


def make_workload(name: str):
    """Return (K, s0, params) for a named workload."""
    w = dict(WORKLOADS[name])
    nx, ny = w["nx"], w["ny"]
    h = 1.0 / nx
    K = lognormal_grf(nx, ny, h, w["sigma2"], w["ell"], w["cov"], w["seed"])
    s0 = np.zeros((ny, nx))
    return K, s0, w
