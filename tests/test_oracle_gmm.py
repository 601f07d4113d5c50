"""Pins of the oracle's Gaussian-mixture refit (oracle/gmm.py): against scikit-learn's EM
from the same start, EM's monotone log-likelihood, recovery of separated clusters, the
initialisation rule on a worked example, and the mixture outputs read back by the
sampler's mixture code."""
import math
import warnings

import numpy as np
import pytest

from oracle import gmm as GM
from oracle import mdn as MD


def _clusters(g, centres, sig, n_each):
    return np.concatenate([c + s * g.standard_normal((n_each, 8)) for c, s in zip(centres, sig)])


def test_em_equals_scikit_learn_from_the_same_start():
    sk = pytest.importorskip("sklearn.mixture")
    g = np.random.default_rng(1)
    centres = g.uniform(0.2, 0.8, (5, 8))
    x = _clusters(g, centres, [0.01, 0.02, 0.005, 0.03, 0.01], 120)
    x = x[g.permutation(len(x))]
    w0, mu0, var0 = GM.init(x, 6)
    w, mu, var, _ = GM.fit(x, n_comp=6, n_iter=25)
    ref = sk.GaussianMixture(n_components=6, covariance_type="diag", weights_init=w0, means_init=mu0,
                             precisions_init=1.0 / var0, reg_covar=1e-6, max_iter=25, tol=0.0)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        ref.fit(x)
    np.testing.assert_allclose(w, ref.weights_, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(mu, ref.means_, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(var, ref.covariances_, rtol=1e-7, atol=1e-13)


def test_em_log_likelihood_never_decreases():
    g = np.random.default_rng(2)
    for trial in range(5):
        x = g.uniform(0, 1, (300, 8)) ** (1 + trial)      # no mixture structure: EM still climbs
        _, _, _, hist = GM.fit(x, n_iter=30)
        d = np.diff(hist)
        assert (d > -1e-9 * np.abs(hist[1:])).all(), d.min()
        assert hist[-1] > hist[0]


def test_em_recovers_separated_clusters():
    g = np.random.default_rng(3)
    centres = np.array([[0.2] * 8, [0.8] * 8, [0.2] * 4 + [0.8] * 4, [0.5] * 8])
    sig = [0.01, 0.02, 0.015, 0.005]
    x = _clusters(g, centres, sig, 400)
    w, mu, var, _ = GM.fit(x, n_comp=4, n_iter=60)
    for c, s in zip(centres, sig):
        j = int(np.argmin(np.abs(mu - c).sum(axis=1)))
        assert np.abs(mu[j] - c).max() < 5 * s / math.sqrt(400)
        assert np.abs(np.sqrt(var[j]) / s - 1).max() < 0.25
        assert abs(w[j] - 0.25) < 1e-3


def test_initialisation_worked_example():
    # five present points (a NaN row is skipped), K = min(16, 5) = 5: ranks floor((k + 1/2) 5 / 5) = k;
    # with K = 2: ranks floor(1.25) = 1 and floor(3.75) = 3 of the f0 (u1) order
    x = np.full((6, 8), 0.5)
    x[:, 1] = [0.9, 0.1, np.nan, 0.5, 0.3, 0.7]
    p = GM.present(x)
    assert p.shape == (5, 8)
    w, mu, var = GM.init(p, 2)
    assert mu[:, 1].tolist() == [0.3, 0.7]
    assert np.allclose(w, 0.5)
    assert np.allclose(var[0, 1], np.var([0.9, 0.1, 0.5, 0.3, 0.7]) + 1e-6) and np.allclose(var[0, 0], 1e-6)
    _, mu5, _ = GM.init(p, 16)
    assert mu5[:, 1].tolist() == [0.1, 0.3, 0.5, 0.7, 0.9]


def test_mixture_outputs_read_back():
    # to_raw -> the sampler's mixture (oracle.mdn.mixture): equal weights over the used components,
    # the fitted means and widths, left-out components at e^-30
    g = np.random.default_rng(4)
    w = np.array([0.5, 0.3, 0.195, 0.005])
    mu = g.uniform(0.1, 0.9, (4, 8))
    var = g.uniform(1e-6, 1e-2, (4, 8))
    raw = GM.to_raw(w, mu, var, min_weight=0.01)
    lpi, m, ls = MD.mixture(raw[None, :])
    pi = np.exp(lpi[0])
    np.testing.assert_allclose(pi[:3], 1 / 3, rtol=1e-10)
    assert (pi[3:] < 1e-12).all()
    np.testing.assert_allclose(m[0, :4], mu, rtol=1e-9)
    np.testing.assert_allclose(np.exp(2 * ls[0, :4]), var, rtol=1e-8)
    # an empty band: 16 equal broad components centred in the box
    lpi, m, ls = MD.mixture(GM.to_raw(np.zeros(0), np.zeros((0, 8)), np.zeros((0, 8)))[None, :])
    np.testing.assert_allclose(np.exp(lpi[0]), 1 / 16, rtol=1e-12)
    assert np.allclose(m, 0.5) and np.allclose(ls, 0.0, atol=1e-6)
