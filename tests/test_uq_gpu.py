"""The batched pCN sampler with the CUDA forward model: R chains, one context of R
realisations per proposal batch; the forward observations of a proposal match the oracle's
Algorithm 1 run on the same permeability, and the chains keep consistent states."""
import numpy as np
import pytest

from oracle import mpm_oracle as O
from paper_2103_11050_gb300 import uq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11050_gb300 import build
    build.build()


def test_pcn_chains_on_the_gpu_forward_model():
    from paper_2103_11050_gb300 import binding as B
    nx = ny = 32
    R, steps, eta, M = 4, 6, 0.05, 3.0
    prior = uq.Prior(nx, ny, 1.0, 0.2)
    s0 = np.zeros((ny, nx))
    cells = np.array([j * nx + nx // 2 for j in range(0, ny, 4)] + [5 * nx + 3, 20 * nx + 10])
    ctx = B.Context(R, nx, ny)
    ctx.set_precision(B.PREC_FP32_IR, 1e-14, 30)
    ctx.set_fluids(M)
    ctx.set_decomposition([16, 16], [16, 16], 4, 1, 1.0)
    fwd = uq.Forward(ctx, s0, eta, steps, cells)
    # synthetic data: the forward model at a reference field, plus noise
    rng = np.random.default_rng(11)
    truth = prior.field(prior.noise(rng))
    sigma = 0.02
    data = fwd(np.stack([truth] * R))[0] + sigma * rng.standard_normal(len(cells))
    ch = uq.start(prior, fwd, data, sigma, R, rng)
    # the forward model of chain 0 against the oracle
    prob = O.Problem(nx, ny, 1.0 / nx, (0, 0, 1, 1), (1.0, 0.0, 0.0, 0.0), M, 1.0)
    dec = O.Decomposition(nx, ny, [16, 16], [16, 16], 4, 1, 1.0)
    K0 = prior.field(ch.xi[0])
    st = O.simulate_init(K0, s0, prob, dec, eta)
    for _ in range(steps):
        O.simulate_step(st, K0, prob, dec, eta, 0.5, 1)
    np.testing.assert_allclose(ch.obs[0], st.s.reshape(-1)[cells], rtol=1e-8, atol=1e-12)
    for _ in range(3):
        uq.pcn_iteration(ch, prior, fwd, data, sigma, 0.2, rng)
    # stored log-likelihoods belong to the stored states (recomputed in one more batch)
    obs = fwd(np.stack([prior.field(x) for x in ch.xi]))
    np.testing.assert_allclose(obs, ch.obs, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(ch.loglik, uq.log_likelihood(obs, data, sigma), rtol=1e-9)
    assert len(ch.history) == 3
    ctx.close()
