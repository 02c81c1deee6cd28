"""Batched Markov chain Monte Carlo over permeability fields (the uncertainty-quantification
setting that motivates the method, Sections 1 and 6): R chains advance together, and every
batch of R proposals is one pass of Algorithm 1 over R realisations in a single context, so
all their local solves, interface solves and downscalings run in the same launches.

Sampler: preconditioned Crank-Nicolson (pCN; Cotter, Roberts, Stuart and White, Statistical
Science 28, 2013) on the white noise xi of the log-permeability field (fields.grf_from_noise):
    xi' = sqrt(1 - beta^2) xi + beta zeta,  zeta ~ N(0, I),
accepted with probability min(1, exp(loglik(xi') - loglik(xi))): the proposal preserves the
Gaussian prior, so only the likelihood ratio enters.  The likelihood compares observations
of the simulated saturation (values at chosen cells after a fixed number of Algorithm 1
steps) with data under independent Gaussian noise of standard deviation sigma.

Only the accept / reject arithmetic (R numbers per iteration) runs on the host; the forward
model is the library's CUDA path.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fields


@dataclass
class Prior:
    """Log-normal permeability prior: K = exp(mean_log + Y), Y a Gaussian random field."""
    nx: int
    ny: int
    sigma2: float
    ell: float
    cov: str = "exponential"
    mean_log: float = 0.0

    def field(self, xi):
        return fields.grf_from_noise(self.nx, self.ny, 1.0 / self.nx, self.sigma2, self.ell, self.cov, xi,
                                     self.mean_log)

    def noise(self, rng):
        return fields.grf_noise(self.nx, self.ny, rng)


@dataclass
class Forward:
    """Algorithm 1 on a context of R realisations: obs[r] = s_r at obs_cells (flat cell indices)
    after n_steps steps from s0, for the permeabilities Ks [R][ny][nx]."""
    ctx: object
    s0: np.ndarray
    eta: float
    n_steps: int
    obs_cells: np.ndarray
    cfl: float = 0.5
    n_sub: int = 1

    def __call__(self, Ks):
        R = Ks.shape[0]
        self.ctx.set_permeability(np.ascontiguousarray(Ks))
        self.ctx.set_saturation(np.ascontiguousarray(np.broadcast_to(self.s0, Ks.shape)))
        self.ctx.init(self.eta)
        for _ in range(self.n_steps):
            self.ctx.step(self.eta, self.cfl, self.n_sub)
        s = self.ctx.get_saturation()
        return s.reshape(R, -1)[:, self.obs_cells]


def log_likelihood(obs, data, sigma):
    """Gaussian log-likelihood (up to a constant) of each row of obs."""
    d = np.asarray(obs) - np.asarray(data)[None, :]
    return -0.5 * np.sum(d * d, axis=1) / (sigma * sigma)


def pcn_accept(ll_old, ll_new, u):
    """Acceptance of pCN proposals: u < exp(ll_new - ll_old), u ~ U[0,1) per chain."""
    return np.log(np.maximum(u, 1e-300)) < (ll_new - ll_old)


@dataclass
class Chains:
    xi: list                       # per chain, the current white noise
    loglik: np.ndarray             # per chain, its log-likelihood
    obs: np.ndarray                # per chain, its observations
    accepted: np.ndarray           # per chain, accepted proposals so far
    history: list = field(default_factory=list)  # per iteration: loglik, accepted flags


def start(prior, forward, data, sigma, R, rng):
    xi = [prior.noise(rng) for _ in range(R)]
    obs = forward(np.stack([prior.field(x) for x in xi]))
    return Chains(xi, log_likelihood(obs, data, sigma), obs, np.zeros(R, dtype=int))


def pcn_iteration(chains, prior, forward, data, sigma, beta, rng):
    """One pCN iteration of every chain: R proposals through one forward batch, then the
    per-chain accept / reject."""
    R = len(chains.xi)
    c = np.sqrt(1.0 - beta * beta)
    prop = [c * x + beta * prior.noise(rng) for x in chains.xi]
    obs = forward(np.stack([prior.field(x) for x in prop]))
    ll = log_likelihood(obs, data, sigma)
    acc = pcn_accept(chains.loglik, ll, rng.random(R))
    for r in range(R):
        if acc[r]:
            chains.xi[r] = prop[r]
            chains.loglik[r] = ll[r]
            chains.obs[r] = obs[r]
    chains.accepted += acc
    chains.history.append({"loglik": chains.loglik.copy(), "accepted": acc.copy(), "proposal_loglik": ll})
    return chains
