"""Pins of the oracle's PSD/foreground module: the per-channel PSD reduces to Eq. psd, the
foreground adds to both channels, and the stretch sampler leaves its target invariant
(prior-only box, and a posterior centred on the truth for noise drawn from known levels)."""
import math

import numpy as np
from scipy import stats

from oracle import constants as OC
from oracle import likelihood as LK
from oracle import psd as PS
from oracle import psdmcmc as PM
from paper_2405_04690_gb300 import synth

F = (3146 + np.arange(0, 2 ** 16, 64)) * OC.DF        # 1024 bins over 0.1-33 mHz


def test_channel_psd_reduces_to_eq_psd_and_adds_the_foreground():
    p = np.array([15e-12, 3e-15, 9e-12, 2e-15, 1e-60, 1.2, 2.8e-3, 1763.3, 1686.3])
    sa, se = PM.channel_psd(F, p)
    np.testing.assert_allclose(sa, PS.psd_ae(F, 15e-12, 3e-15), rtol=1e-14)
    np.testing.assert_allclose(se, PS.psd_ae(F, 9e-12, 2e-15), rtol=1e-14)
    p[4] = 3.3e-44
    sa2, se2 = PM.channel_psd(F, p)
    fg = PS.foreground_ae(F, 3.3e-44, 1.2, 2.8e-3, 1763.3, 1686.3)
    np.testing.assert_allclose(sa2 - sa, fg, rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(se2 - se, fg, rtol=1e-10, atol=1e-300)
    # likelihood with equal channels = Eq. like with one shared PSD
    g = np.random.default_rng(1)
    r = synth.unit_complex_normal(g, (2, len(F))) * np.sqrt(sa2 / (4 * OC.DF))
    q = p.copy()
    q[2], q[3] = q[0], q[1]
    assert abs(PM.loglike(r, F, OC.DF, q) - LK.loglike(r, PM.channel_psd(F, q)[0], OC.DF)) < 1e-9 * abs(
        LK.loglike(r, PM.channel_psd(F, q)[0], OC.DF))


def _box():
    lo = np.array([math.log(5e-12), math.log(1e-15), math.log(5e-12), math.log(1e-15), math.log(1e-45), 0.8, 1e-3,
                   500.0, 500.0])
    hi = np.array([math.log(45e-12), math.log(9e-15), math.log(45e-12), math.log(9e-15), math.log(1e-42), 1.6, 4e-3,
                   3000.0, 3000.0])
    return lo, hi


def test_prior_only_stretch_sampler_keeps_the_box_uniform():
    # beta = 0 at both temperatures: the target is the uniform box in v, for which an
    # ensemble of independent uniform draws is stationary. 60 ensembles started from exact
    # draws run 6 sweeps; the final positions must still be uniform in every coordinate
    # (dropping the z^(d-1) factor, planted in the oracle on the CPU, fails this).
    lo, hi = _box()
    T, W = 2, 16
    g = np.random.default_rng(2)
    f = F[:16]
    resid = np.zeros((W, 2, len(f)), complex)
    final = []
    for e in range(60):
        cfg = PM.PsdConfig(T, W, lo, hi, betas=[0.0, 0.0], key=(7, e))
        v = lo + (hi - lo) * g.uniform(size=(T, W, 9))
        params = np.array([[PM.from_v(v[t, w]) for w in range(W)] for t in range(T)])
        logl = np.zeros((T, W))
        for s in range(6):
            PM.sweep(cfg, params, logl, resid, f, OC.DF, s)
        final.extend((np.array([PM.to_v(p) for p in params.reshape(-1, 9)]) - lo) / (hi - lo))
    final = np.asarray(final)
    for d in range(9):
        assert stats.kstest(final[:, d], "uniform").pvalue > 1e-3, d


def test_stretch_sampler_recovers_the_noise_levels():
    # noise drawn from known per-channel levels and a foreground; beta = 1; the walkers'
    # mean of ln sqrt(S_oms,A) and ln sqrt(S_acc,E) lands within 4 posterior sigma of the truth
    lo, hi = _box()
    truth = np.array([15e-12, 3e-15, 12e-12, 4e-15, 3.3e-44, 1.2, 2.8e-3, 1763.3, 1686.3])
    f = (3146 + np.arange(0, 2 ** 17, 128)) * OC.DF
    g = np.random.default_rng(3)
    sa, se = PM.channel_psd(f, truth)
    r = np.stack([synth.unit_complex_normal(g, len(f)) * np.sqrt(sa / (4 * OC.DF)),
                  synth.unit_complex_normal(g, len(f)) * np.sqrt(se / (4 * OC.DF))])
    T, W = 1, 16
    cfg = PM.PsdConfig(T, W, lo, hi, betas=[1.0], key=(3, 4))
    v0 = PM.to_v(truth)
    params = np.array([[PM.from_v(np.clip(v0 + 0.02 * (hi - lo) * g.standard_normal(9), lo, hi))
                        for _ in range(W)]])
    resid = np.stack([r] * W)
    logl = np.array([[PM.loglike(r, f, OC.DF, params[0, w]) for w in range(W)]])
    samples = []
    for s in range(200):
        PM.sweep(cfg, params, logl, resid, f, OC.DF, s)
        if s >= 100:
            samples.extend([PM.to_v(p) for p in params[0]])
    samples = np.asarray(samples)
    for d in (0, 3):
        m, sd = samples[:, d].mean(), samples[:, d].std()
        assert sd > 0 and abs(m - v0[d]) < 4 * sd + 1e-3, (d, m, v0[d], sd)
