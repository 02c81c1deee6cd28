"""The seeded synthetic inputs (paper_2103_11050_gb300/fields.py) have the structure their
recipes state: log-normal fields with the requested log-variance, binary channelised fields
at the requested coverage and contrast, the fingering inlet, the uneven decompositions, and
reproducibility from the seed.  CPU only."""
import numpy as np

from paper_2103_11050_gb300 import fields


def test_lognormal_field_statistics_and_seed():
    n, s2, ell = 256, 2.0, 0.02
    K = fields.lognormal_grf(n, n, 1.0 / n, s2, ell, "exponential", seed=7)
    assert K.shape == (n, n) and K.dtype == np.float64 and K.flags["C_CONTIGUOUS"] and np.all(K > 0)
    Y = np.log(K)
    # correlation length small against the domain: the sample moments are close to the model's
    assert abs(Y.mean()) < 0.2 * np.sqrt(s2)
    assert 0.8 * s2 < Y.var() < 1.2 * s2
    assert np.array_equal(K, fields.lognormal_grf(n, n, 1.0 / n, s2, ell, "exponential", seed=7))
    assert not np.array_equal(K, fields.lognormal_grf(n, n, 1.0 / n, s2, ell, "exponential", seed=8))
    # the Gaussian covariance gives a smoother field: smaller neighbour differences
    G = np.log(fields.lognormal_grf(n, n, 1.0 / n, s2, 0.05, "gaussian", seed=7))
    E = np.log(fields.lognormal_grf(n, n, 1.0 / n, s2, 0.05, "exponential", seed=7))
    assert np.mean(np.diff(G, axis=1) ** 2) < np.mean(np.diff(E, axis=1) ** 2)


def test_field_is_linear_in_its_noise():
    # the sampler's parametrisation: log K is a linear map of the white noise
    n = 32
    rng = np.random.default_rng(3)
    a, b = fields.grf_noise(n, n, rng), fields.grf_noise(n, n, rng)
    la = np.log(fields.grf_from_noise(n, n, 1.0 / n, 1.0, 0.1, "exponential", a))
    lb = np.log(fields.grf_from_noise(n, n, 1.0 / n, 1.0, 0.1, "exponential", b))
    lab = np.log(fields.grf_from_noise(n, n, 1.0 / n, 1.0, 0.1, "exponential", 2.0 * a - b))
    np.testing.assert_allclose(lab, 2.0 * la - lb, atol=1e-12)


def test_channelised_field():
    K = fields.channelised(256, 256, 1.0, 1e-4, 0.30, (8, 24), seed=3)
    vals = np.unique(K)
    assert vals.tolist() == [1e-4, 1.0]
    cover = np.mean(K == 1.0)
    assert 0.30 <= cover < 0.45
    # channels run along x: most columns cut every channel, so each column holds channel cells
    assert np.all(np.any(K == 1.0, axis=0))
    assert np.array_equal(K, fields.channelised(256, 256, 1.0, 1e-4, 0.30, (8, 24), seed=3))


def test_fingering_initial_saturation():
    s0 = fields.fingering_s0(512, 512, 0.05, 8, 0.01, seed=5)
    n_in = round(0.05 * 512)
    assert np.all(s0[:, :n_in] == 1.0)
    noise = s0[:, n_in:n_in + 8]
    assert np.all((noise >= 0.0) & (noise < 0.01)) and noise.std() > 0
    assert np.all(s0[:, n_in + 8:] == 0.0)


def test_uneven_decomposition_and_ensemble():
    parts = (8, 8, 12, 12, 16, 16, 16, 20, 20)
    cw = fields.uneven_widths(128, parts, 11)
    assert sorted(cw) == sorted(parts) and sum(cw) == 128 and cw == fields.uneven_widths(128, parts, 11)
    Ks, s0, cw2, rh2, w = fields.make_ensemble(R=3)
    assert Ks.shape == (3, 128, 128) and np.all(s0 == 0.0) and cw2 == cw
    assert sorted(rh2) == sorted(parts)
    # the first realisations do not depend on how many are drawn
    Ks5 = fields.make_ensemble(R=5)[0]
    assert np.array_equal(Ks5[:3], Ks)
    assert not np.array_equal(Ks[0], Ks[1])
