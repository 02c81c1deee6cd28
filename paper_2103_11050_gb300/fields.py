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


def _embedding_spectrum(nx, ny, h, sigma2, ell, cov):
    """Eigenvalues of the circulant embedding of the covariance on the 2nx x 2ny periodic grid
    (negative ones clipped to zero)."""
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
    return np.clip(lam, 0.0, None)


def grf_from_noise(nx: int, ny: int, h: float, sigma2: float, ell: float, cov: str, xi: np.ndarray,
                   mean_log: float = 0.0) -> np.ndarray:
    """K = exp(mean_log + Y) for the white noise xi (complex, [2ny][2nx], real and imaginary
    parts independent standard normals): Y is the real part of the circulant-embedding
    synthesis, restricted to the grid.  A linear map of xi, so a Gaussian prior on xi is the
    field's prior (the parametrisation a sampler over permeabilities moves in)."""
    mx, my = 2 * nx, 2 * ny
    lam = _embedding_spectrum(nx, ny, h, sigma2, ell, cov)
    y = np.fft.fft2(np.sqrt(lam / (mx * my)) * xi)
    return np.ascontiguousarray(np.exp(mean_log + y.real[:ny, :nx]))


def grf_noise(nx: int, ny: int, rng) -> np.ndarray:
    """The white noise of grf_from_noise, drawn from rng."""
    mx, my = 2 * nx, 2 * ny
    return rng.standard_normal((my, mx)) + 1j * rng.standard_normal((my, mx))


def lognormal_grf(nx: int, ny: int, h: float, sigma2: float, ell: float,
                  cov: str = "exponential", seed: int = 0,
                  mean_log: float = 0.0) -> np.ndarray:
    """K = exp(mean_log + Y), Y a zero-mean GRF with the named covariance."""
    rng = np.random.default_rng(seed)
    return grf_from_noise(nx, ny, h, sigma2, ell, cov, grf_noise(nx, ny, rng), mean_log)


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


# Workloads used by the tests and the benchmark: grid, subdomain layout, permeability recipe,
# viscosity ratio, rebuild threshold and trajectory length of each, listed per entry.
# field: "grf" (log-normal, covariance / variance / correlation length / seed),
# "channelised" (binary channels: k_channel, k_matrix, coverage, width range, seed),
# "homogeneous" (K = 1).  s0: "zero" (oil-filled) or "fingering" (fingering_s0).
WORKLOADS = {
    # 64x64, 4x4 subdomains of 16x16, exponential GRF (ell 0.1, var 1), M = 1,
    # rebuild every step (eta < 0).
    "gaussian64": dict(nx=64, ny=64, ncx=4, ncy=4, field="grf", sigma2=1.0, ell=0.1, cov="exponential",
                       seed=1, M=1.0, eta=-1.0, steps=20),
    # 256x256, 16x16 subdomains, Gaussian covariance (ell 0.05, var 4), M = 5, eta = 0.1.
    "gaussian256": dict(nx=256, ny=256, ncx=16, ncy=16, field="grf", sigma2=4.0, ell=0.05, cov="gaussian",
                        seed=2, M=5.0, eta=0.1, steps=500),
    # 1024x1024, 64x64 subdomains of 16x16; binary K in {1, 1e-4}: sinusoidal channels along x,
    # widths 8..24 cells, added until 30 % of the cells are channel (contrast 1e4); M = 5,
    # eta = 0.1 (the values of the 256^2 workload).
    "channel1024": dict(nx=1024, ny=1024, ncx=64, ncy=64, field="channelised", k_channel=1.0, k_matrix=1e-4,
                        coverage=0.30, widths=(8, 24), seed=3, M=5.0, eta=0.1, steps=500),
    # 512x512, 32x32 subdomains of 16x16, K = 1, M = 10, water-filled inlet strip (x < 0.05) with
    # 1 % seeded noise in the next 8 columns; eta = 0.1 (the runs also take 0.05 and 0.2).
    "finger512": dict(nx=512, ny=512, ncx=32, ncy=32, field="homogeneous", s0="fingering", seed=5, M=10.0,
                      eta=0.1, steps=5000),
}

# The ensemble workload: R independent realisations of a log-normal field (exponential
# covariance, variance 2, correlation length drawn uniformly in [0.05, 0.2] per realisation
# with a generator of seed ``seed``, field seed seed + r), all on one uneven tensor-product
# decomposition whose column widths / row heights are seeded permutations of
# 8, 8, 12, 12, 16, 16, 16, 20, 20 (sum 128).
ENSEMBLE = dict(nx=128, ny=128, R=256, parts=(8, 8, 12, 12, 16, 16, 16, 20, 20), col_seed=11, row_seed=12,
                sigma2=2.0, ell_range=(0.05, 0.2), cov="exponential", seed=4, M=3.0, eta=0.05, steps=500)


def make_ensemble(R: int | None = None, **over):
    """(Ks [R][ny][nx], s0 [ny][nx], col_w, row_h, params) of the ensemble workload; the first
    R realisations are the same whatever R is."""
    w = dict(ENSEMBLE)
    w.update(over)
    R = w["R"] if R is None else int(R)
    nx, ny = w["nx"], w["ny"]
    ells = np.random.default_rng(w["seed"]).uniform(w["ell_range"][0], w["ell_range"][1], max(R, w["R"]))
    Ks = np.stack([lognormal_grf(nx, ny, 1.0 / nx, w["sigma2"], ells[r], w["cov"], w["seed"] + r) for r in range(R)])
    cw = uneven_widths(nx, w["parts"], w["col_seed"])
    rh = uneven_widths(ny, w["parts"], w["row_seed"])
    return Ks, np.zeros((ny, nx)), cw, rh, w


def make_workload(name: str):
    """Return (K, s0, params) for a named workload."""
    w = dict(WORKLOADS[name])
    nx, ny = w["nx"], w["ny"]
    h = 1.0 / nx
    kind = w.get("field", "grf")
    if kind == "grf":
        K = lognormal_grf(nx, ny, h, w["sigma2"], w["ell"], w["cov"], w["seed"])
    elif kind == "channelised":
        K = channelised(nx, ny, w["k_channel"], w["k_matrix"], w["coverage"], w["widths"], w["seed"])
    elif kind == "homogeneous":
        K = np.ones((ny, nx))
    else:
        raise ValueError(f"unknown field kind {kind!r}")
    if w.get("s0", "zero") == "fingering":
        s0 = fingering_s0(nx, ny, 0.05, 8, 0.01, seed=w["seed"])
    else:
        s0 = np.zeros((ny, nx))
    return K, s0, w
