"""Pins of the oracle's mixture-density proposal: gradients against finite differences,
exact normalisation of the truncated mixture, sampling against the density, the unit-box
coordinate map, and Adam's first step."""
import math

import numpy as np
from scipy import integrate, stats
from scipy.special import ndtr

from oracle import mdn as MD

from _sweep_setup import small_ensemble


def _small_theta(g):
    return MD.init_params(g, scale=0.5)


def _sigma_logits(k):
    return np.arange(k * 17 + 9, k * 17 + 17)


def _broad_raw(g, rows, shift=2.0):
    raw = g.normal(0, 1, (rows, MD.N_OUT))
    for k in range(MD.N_COMP):
        raw[:, _sigma_logits(k)] += shift        # sigma ~ 0.1-0.5: smooth enough for the checks
    return raw


def test_grad_raw_matches_finite_differences():
    # fourth-order central differences of -ln q
    g = np.random.default_rng(1)
    raw = _broad_raw(g, 3, shift=1.0)
    u = g.uniform(0.05, 0.95, (3, MD.N_DIM))
    an = MD.grad_raw(raw, u)
    h = 1e-4
    for j in g.choice(MD.N_OUT, 80, replace=False):
        f = []
        for step in (h, -h, 2 * h, -2 * h):
            r = raw.copy()
            r[:, j] += step
            f.append(-MD.log_q(r, u))
        fd = (8 * (f[0] - f[1]) - (f[2] - f[3])) / (12 * h)
        np.testing.assert_allclose(an[:, j], fd, rtol=1e-7, atol=1e-9)


def test_backward_matches_finite_differences():
    g = np.random.default_rng(2)
    theta = _small_theta(g)
    x = g.normal(0, 1, (4, MD.N_IN))
    u = g.uniform(0.05, 0.95, (4, MD.N_DIM))
    grad = MD.backward(theta, x, u)
    assert grad.shape == (MD.n_params(),)
    # parameters spread over every layer's weights and biases
    offs, k = [], 0
    for o, i in MD.LAYERS:
        offs.append((k, o * i))
        k += o * i
        offs.append((k, o))
        k += o
    eps = 1e-6
    for start, size in offs:
        for j in g.choice(size, 4, replace=False):
            idx = start + j
            tp, tm = theta.copy(), theta.copy()
            tp[idx] += eps
            tm[idx] -= eps
            fd = (MD.nll(tp, x, u) - MD.nll(tm, x, u)) / (2 * eps)
            assert abs(grad[idx] - fd) <= 1e-5 * max(1e-3, abs(fd)), (idx, grad[idx], fd)


def test_truncated_normal_integrates_to_one_on_the_box():
    for mu, ls in ((0.02, -3.0), (0.5, 0.0), (0.97, -1.0), (0.3, -8.0)):
        f = lambda x: math.exp(MD.log_trunc_normal(np.array(x), np.array(mu), np.array(ls)))
        val, _ = integrate.quad(f, 0.0, 1.0, points=[mu], limit=200)
        assert abs(val - 1.0) < 1e-7, (mu, ls, val)


def test_mixture_density_integrates_to_one():
    # broad random mixture; Monte Carlo over the unit box
    g = np.random.default_rng(3)
    raw = _broad_raw(g, 1, shift=3.0)
    u = g.uniform(0, 1, (400000, MD.N_DIM))
    q = np.exp(MD.log_q(np.repeat(raw, len(u), axis=0), u))
    est = q.mean()
    err = q.std() / math.sqrt(len(u))
    assert abs(est - 1.0) < 5 * err + 1e-3, (est, err)


def test_sampling_follows_the_density():
    g = np.random.default_rng(4)
    raw = g.normal(0, 1, (1, MD.N_OUT))
    lpi, mu, ls = MD.mixture(raw)
    draws = MD.sample(np.repeat(raw, 20000, axis=0), g)
    # marginal CDF of dimension 2 under the mixture, by its closed form
    d = 2

    def cdf(x):
        s = np.exp(ls[0, :, d])
        m = mu[0, :, d]
        lo, hi = ndtr(-m / s), ndtr((1 - m) / s)
        return float(np.sum(np.exp(lpi[0]) * (ndtr((x - m) / s) - lo) / (hi - lo)))

    assert stats.kstest(draws[:, d], np.vectorize(cdf)).pvalue > 1e-3


def test_unit_coordinates_round_trip():
    cfg, state, _, _ = small_ensemble(seed=12)
    g = np.random.default_rng(5)
    for _ in range(20):
        u = g.uniform(0, 1, MD.N_DIM)
        th = MD.from_unit(cfg, 1, u)
        np.testing.assert_allclose(MD.to_unit(cfg, 1, th), u, rtol=1e-10, atol=1e-12)


def test_adam_first_step_moves_by_lr_times_sign():
    theta = np.array([1.0, -2.0, 0.5])
    grad = np.array([3.0, -0.2, 1e-3])
    t, m, v = MD.adam(theta, np.zeros(3), np.zeros(3), grad, 1, 0.01)
    np.testing.assert_allclose(t, theta - 0.01 * np.sign(grad), rtol=0, atol=1e-6)


def raw_from(pi, mu, s):
    """Raw network outputs [272] for given weights pi [16], means mu [16][8] and widths s [16][8]."""
    raw = np.empty((MD.N_COMP, 1 + 2 * MD.N_DIM))
    raw[:, 0] = np.log(pi)
    raw[:, 1:1 + MD.N_DIM] = np.log(mu / (1 - mu))
    sg = (np.log(s) - MD.S_MIN) / (MD.S_MAX - MD.S_MIN)
    raw[:, 1 + MD.N_DIM:] = np.log(sg / (1 - sg))
    return raw.ravel()


def _peaked_raw(g):
    pi = g.dirichlet(np.ones(MD.N_COMP))
    mu = g.uniform(0.2, 0.8, (MD.N_COMP, MD.N_DIM))
    s = g.uniform(0.03, 0.15, (MD.N_COMP, MD.N_DIM))
    return raw_from(pi, mu, s)


def test_raw_from_inverts_the_output_maps():
    g = np.random.default_rng(11)
    pi = g.dirichlet(np.ones(MD.N_COMP))
    mu = g.uniform(0.1, 0.9, (MD.N_COMP, MD.N_DIM))
    s = g.uniform(0.01, 0.5, (MD.N_COMP, MD.N_DIM))
    lpi, m2, ls = MD.mixture(raw_from(pi, mu, s)[None, :])
    assert np.allclose(np.exp(lpi[0]), pi, rtol=1e-12)
    assert np.allclose(m2[0], mu, rtol=1e-12)
    assert np.allclose(np.exp(ls[0]), s, rtol=1e-12)


def test_draw_unit_follows_the_mixture_marginals():
    # Draws from fixed words: each coordinate's empirical CDF against the mixture's
    # closed-form marginal CDF sum_k pi_k [Phi((x-mu)/s) - Phi(-mu/s)] / Z_k.
    g = np.random.default_rng(12)
    raw = _peaked_raw(g)
    lpi, mu, ls = MD.mixture(raw[None, :])
    pi, mu, s = np.exp(lpi[0]), mu[0], np.exp(ls[0])
    n = 4000
    words = g.integers(0, 2 ** 32, (n, 9), dtype=np.uint64)
    u = np.array([MD.draw_unit(raw, int(wd[0]), [int(x) for x in wd[1:]]) for wd in words])
    for d in (0, 3, 7):
        def cdf(x, d=d):
            x = np.atleast_1d(x)[:, None]
            lo, hi = ndtr(-mu[:, d] / s[:, d]), ndtr((1 - mu[:, d]) / s[:, d])
            return np.sum(pi * (ndtr((x - mu[:, d]) / s[:, d]) - lo) / (hi - lo), axis=1)
        assert stats.kstest(u[:, d], cdf).pvalue > 1e-3


def test_defensive_density_integrates_to_one_and_reduces_to_prior():
    g = np.random.default_rng(13)
    raw = _peaked_raw(g)
    # the integral of q over the box is 1: E_uniform[q] for a mixture broad enough that
    # uniform draws sample it well
    pi = g.dirichlet(np.ones(MD.N_COMP))
    broad = raw_from(pi, g.uniform(0.2, 0.8, (MD.N_COMP, MD.N_DIM)), g.uniform(0.25, 0.6, (MD.N_COMP, MD.N_DIM)))
    x = g.uniform(0, 1, (20000, MD.N_DIM))
    q = np.exp(MD.log_q(np.tile(broad, (len(x), 1)), x))
    assert abs(q.mean() - 1.0) < 5 * q.std() / math.sqrt(len(x)), (q.mean(), q.std())
    # eps = 1 is the prior (density 1 everywhere); eps mixes linearly
    x = g.uniform(0, 1, MD.N_DIM)
    assert MD.log_q_defensive(raw, x, 1.0) == 0.0
    q = math.exp(MD.log_q(raw[None, :], x[None, :])[0])
    assert abs(math.exp(MD.log_q_defensive(raw, x, 0.25)) - (0.25 + 0.75 * q)) < 1e-12 * (1 + q)


def test_to_bf16_matches_torch_rounding():
    # round to nearest, ties to even, including exact ties and values near overflow
    torch = __import__("pytest").importorskip("torch")
    g = np.random.default_rng(14)
    x = np.concatenate([g.normal(0, 1, 20000), g.normal(0, 1e-30, 1000), g.normal(0, 1e30, 1000)])
    ties = (np.arange(1, 2000, dtype=np.uint32) << 16 | 0x8000).view(np.float32).astype(np.float64)
    x = np.concatenate([x, ties, -ties])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(MD.to_bf16(x), want)


def test_quantized_network_is_the_rounded_one():
    # quantized forward = plain forward of bf16-rounded weights when the hidden
    # activations happen to be representable; in general it stays within the bf16
    # error bound of the plain network
    g = np.random.default_rng(15)
    theta = MD.init_params(g)
    x = MD.to_bf16(g.normal(0, 1, (64, MD.N_IN)))
    rq, aq = MD.forward(theta, x, quantized=True)
    for a in aq[1:-1]:
        assert np.array_equal(a, MD.to_bf16(a))
    r0, _ = MD.forward(theta, x)
    assert np.linalg.norm(rq - r0) / np.linalg.norm(r0) < 2e-2
    # layer by layer: the first hidden layer is relu(x bf16(W1)^T + b1), rounded
    layers = MD.unpack(theta)
    h1 = MD.to_bf16(np.maximum(x @ MD.to_bf16(layers[0][0]).T + layers[0][1], 0))
    assert np.array_equal(aq[1], h1)


def test_features_whiten_the_band_and_interleave_re_im():
    # noise drawn as z sqrt(S_n / (4 df)) (z unit complex normal) whitens back to z exactly:
    # x[ch 512 + 2 i] = Re z[ch][nb + i], x[ch 512 + 2 i + 1] = Im z[ch][nb + i] for the band's
    # own sub-band (the middle third of the window); the neighbours do not enter
    from oracle import constants as OC
    from oracle import psd as OP
    from paper_2405_04690_gb300 import synth
    nb = 256
    k0 = int(2.2e-3 * OC.TOBS)
    f = (k0 + np.arange(3 * nb)) * OC.DF
    s = OP.psd_ae(f, OC.SQRT_S_OMS, OC.SQRT_S_ACC)
    z = synth.unit_complex_normal(synth.rng(12), (2, 3 * nb))
    rho = z * np.sqrt(s / (4 * OC.DF))
    x = MD.features(rho, s, OC.DF, nb)
    assert x.shape == (4 * nb,)
    for ch in range(2):
        np.testing.assert_allclose(x[ch * 2 * nb:(ch + 1) * 2 * nb:2], z[ch, nb:2 * nb].real, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(x[ch * 2 * nb + 1:(ch + 1) * 2 * nb:2], z[ch, nb:2 * nb].imag, rtol=1e-13,
                                   atol=1e-13)
    rho2 = rho.copy()
    rho2[:, :nb] *= 7.0
    rho2[:, 2 * nb:] = 0.0
    assert np.array_equal(MD.features(rho2, s, OC.DF, nb), x)
    # on whitened noise the Eq. inner weight gives <n|n> = sum x^2 per channel ~ 2 per bin
    assert abs(np.sum(x ** 2) / (2 * nb) - 2.0) < 5 * 2.0 / math.sqrt(2 * nb)
