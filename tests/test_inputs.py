"""The seeded input recipe (paper_2405_04690_gb300/synth.py) draws what it states: the prior
distributions of the 8 source parameters, the noise normalisation, the per-walker PSD amplitudes
and seed reproducibility. The GPU path and the oracle both read these inputs, so a drift here
would move both sides together; these checks hold the recipe itself."""
import math

import numpy as np
from scipy import stats

from oracle import constants as OC
from oracle import mcmc as OM
from paper_2405_04690_gb300 import synth


def test_source_draws_follow_the_recipe():
    g = synth.rng(1000)
    n = 20000
    p = synth.draw_sources(g, n)
    assert p.shape == (8, n) and p.dtype == np.float64
    ks = lambda x, lo, hi: stats.kstest((x - lo) / (hi - lo), "uniform").pvalue
    assert ks(p[1], 1e-3, 4e-3) > 1e-3
    assert ks(np.log10(p[0]), -23.0, -21.5) > 1e-3
    assert ks(p[3], 0.0, 2 * math.pi) > 1e-3 and ks(p[4], 0.0, math.pi) > 1e-3
    assert ks(p[5], -1.0, 1.0) > 1e-3 and ks(p[6], -1.0, 1.0) > 1e-3
    assert ks(p[7], 0.0, 2 * math.pi) > 1e-3
    # fdot from the GR chirp: the chirp mass recovered by the oracle's own inverse map is
    # uniform on [0.3, 0.8] solar masses
    mc = np.array([OM.chirp_mass(p[1, i], p[2, i]) for i in range(2000)])
    assert ks(mc, 0.3, 0.8) > 1e-3
    assert (p[2] > 0).all()


def test_log_uniform_frequencies_of_the_uneven_workload():
    g = synth.rng(1002)
    p = synth.draw_sources(g, 20000, 3e-4, 2e-2, log_f=True)
    lo, hi = math.log(3e-4), math.log(2e-2)
    assert stats.kstest((np.log(p[1]) - lo) / (hi - lo), "uniform").pvalue > 1e-3
    # the octave shares of the band lengths: N = 128 below 1 mHz, 256 for 1-2, 512 for 2-4,
    # 1024 above (log-uniform over 0.3-20 mHz gives 28.7, 16.5, 16.5 and 38.3 %)
    want = np.diff(np.log([3e-4, 1e-3, 2e-3, 4e-3, 2e-2])) / (hi - lo)
    got = np.histogram(p[1], [3e-4, 1e-3, 2e-3, 4e-3, 2e-2])[0] / p.shape[1]
    assert np.abs(got - want).max() < 0.015
    np.testing.assert_allclose(want, [0.287, 0.165, 0.165, 0.383], atol=1e-3)


def test_noise_and_psd_amplitudes():
    g = synth.rng(1003)
    z = synth.unit_complex_normal(g, (2, 200000))
    # Re and Im independent N(0, 1): E|z|^2 = 2, so scaled by sqrt(S / (4 df)) the noise gives
    # E<n|n> = 4 df sum |n|^2 / S = 2 per bin and channel
    m = (np.abs(z) ** 2).mean()
    assert abs(m - 2.0) < 5 * 2.0 / math.sqrt(z.size)
    assert abs(np.mean(z.real * z.imag)) < 5 / math.sqrt(z.size)
    a = synth.draw_psd_params(g, 5000)
    r = np.log10(a / np.array([synth.SQRT_S_OMS, synth.SQRT_S_ACC]))
    assert (np.abs(r) <= 0.5).all()
    assert stats.kstest((r[:, 0] + 0.5), "uniform").pvalue > 1e-3
    assert stats.kstest((r[:, 1] + 0.5), "uniform").pvalue > 1e-3
    # the recipe's constants are the ones the oracle uses
    assert synth.TOBS == OC.TOBS and synth.SQRT_S_OMS == OC.SQRT_S_OMS and synth.SQRT_S_ACC == OC.SQRT_S_ACC


def test_draws_are_reproducible_from_the_seed():
    a = synth.draw_sources(synth.rng(7), 64)
    b = synth.draw_sources(synth.rng(7), 64)
    c = synth.draw_sources(synth.rng(8), 64)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
