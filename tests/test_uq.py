"""Host logic of the batched pCN sampler (paper_2103_11050_gb300/uq.py) with stand-in forward
models (no GPU): acceptance rule, state bookkeeping, and invariance of the prior when the
likelihood is flat."""
import numpy as np

from paper_2103_11050_gb300 import uq


def _prior():
    return uq.Prior(8, 8, 1.0, 0.3)


def test_accept_rule():
    ll_old = np.array([-1.0, -1.0, -5.0])
    ll_new = np.array([-2.0, -0.5, -5.0 - np.log(2.0)])
    # accepted iff u < exp(ll_new - ll_old): exp(-1) = 0.37, exp(0.5) > 1, 0.5
    acc = uq.pcn_accept(ll_old, ll_new, np.array([0.36, 0.99, 0.51]))
    assert acc.tolist() == [True, True, False]


def test_flat_likelihood_accepts_everything_and_keeps_the_prior():
    # observations independent of the field: every proposal is accepted, and pCN then leaves
    # the white noise standard normal (its defining property)
    prior = _prior()
    rng = np.random.default_rng(3)
    fwd = lambda Ks: np.zeros((Ks.shape[0], 2))  # noqa: E731
    ch = uq.start(prior, fwd, np.zeros(2), 1.0, 16, rng)
    for _ in range(40):
        uq.pcn_iteration(ch, prior, fwd, np.zeros(2), 1.0, 0.5, rng)
    assert np.all(ch.accepted == 40)
    x = np.concatenate([np.concatenate([v.real.ravel(), v.imag.ravel()]) for v in ch.xi])
    assert abs(np.mean(x)) < 0.05 and abs(np.var(x) - 1.0) < 0.05


def test_rejected_proposals_leave_the_chain_unchanged():
    prior = _prior()
    rng = np.random.default_rng(4)
    cells = np.array([0, 9, 27, 63])
    fwd = lambda Ks: np.log(Ks.reshape(Ks.shape[0], -1)[:, cells])  # noqa: E731
    data = np.zeros(4)
    ch = uq.start(prior, fwd, data, 1e-3, 6, rng)
    for _ in range(5):
        before = [x.copy() for x in ch.xi]
        uq.pcn_iteration(ch, prior, fwd, data, 1e-3, 0.3, rng)
        acc = ch.history[-1]["accepted"]
        for r in range(6):
            if not acc[r]:
                assert np.array_equal(ch.xi[r], before[r])
        # the stored log-likelihoods are those of the stored states
        obs = fwd(np.stack([prior.field(x) for x in ch.xi]))
        np.testing.assert_allclose(ch.loglik, uq.log_likelihood(obs, data, 1e-3), rtol=1e-12)
