"""Small seeded ensemble for the sweep tests (built with the oracle and synth only)."""
import math

import numpy as np

from oracle import constants as OC
from oracle import mcmc as OM
from oracle import psd as OP
from oracle import residual as OR
from oracle import waveform as OW
from paper_2405_04690_gb300 import synth

FRAC = 98
NB = 256


def small_ensemble(seed=0, n_temps=3, n_walkers=2, n_bands=4, n_max=4, n_per_band=2, betas=(1.0, 0.3, 0.0),
                   f_center=2.0e-3, log_occ_odds=0.0, noise=True):
    g = synth.rng(seed)
    band_k0 = int(math.floor(f_center * OC.TOBS))
    k0 = band_k0 - 2 * NB
    n_bins = (n_bands + 4) * NB
    f = (k0 + np.arange(n_bins)) * OC.DF
    s = OP.psd_ae(f, OC.SQRT_S_OMS, OC.SQRT_S_ACC)
    sigma = [0.05, 0.1 * OC.DF, 0.005 * OC.DF / OC.TOBS, 0.05, 0.05, 0.02, 0.02, 0.02]
    cfg = OM.SweepConfig(tobs=OC.TOBS, k0=k0, n_bins=n_bins, band_k0=band_k0, nb=NB, n_bands=n_bands,
                         n_temps=n_temps, n_walkers=n_walkers, n_max=n_max, frac_bits=FRAC,
                         betas=np.tile(np.asarray(betas[:n_temps], dtype=np.float64), (n_bands, 1)),
                         psd=np.tile(s, (n_walkers, 1)), sigma=sigma, log_occ_odds=log_occ_odds,
                         key=(0x1234, 0x5678), f_min=1e-3, f_max=4e-3)
    # truth: n_per_band sources inside each band's own bins, louder than typical
    truth = []
    for b in range(n_bands):
        lo, hi = cfg.band_bins(b)
        p = synth.draw_sources(g, n_per_band, (lo + 10) / OC.TOBS, (hi - 10) / OC.TOBS)
        p[0] = 10.0 ** g.uniform(-22.3, -21.7, n_per_band)
        truth.append(p)
    data = np.zeros((2, n_bins), complex)
    if noise:
        data += synth.unit_complex_normal(g, (2, n_bins)) * np.sqrt(s / (4 * OC.DF))
    for b in range(n_bands):
        for i in range(n_per_band):
            data += _place(cfg, truth[b][:, i])
    params = np.zeros((n_temps, n_walkers, n_bands, n_max, 8))
    exists = np.zeros((n_temps, n_walkers, n_bands, n_max), dtype=bool)
    jit = np.array([0.02, 0.02 * OC.DF, 0.0, 0.02, 0.02, 0.01, 0.01, 0.01])
    for t in range(n_temps):
        for w in range(n_walkers):
            for b in range(n_bands):
                for i in range(n_per_band):
                    th = truth[b][:, i] + jit * g.standard_normal(8)
                    th[0] = truth[b][0, i] * math.exp(0.02 * g.standard_normal())
                    th[5] = min(max(th[5], -1.0), 1.0)
                    th[6] = min(max(th[6], -1.0), 1.0)
                    th[3] %= 2 * math.pi
                    th[4] %= math.pi
                    th[7] %= 2 * math.pi
                    params[t, w, b, i] = th
                    exists[t, w, b, i] = True
    dfix = OR.to_fixed(data, FRAC)
    state = {"params": params, "exists": exists, "resid": cold_residual(cfg, dfix, params, exists)}
    return cfg, state, dfix, s


def cold_residual(cfg, dfix, params, exists):
    """Fixed-point residual of every walker: data minus its cold-chain sources."""
    resid = np.empty((cfg.n_walkers, 2, cfg.n_bins, 2), dtype=np.int64)
    for w in range(cfg.n_walkers):
        r = dfix.copy()
        for b in range(cfg.n_bands):
            for i in range(cfg.n_max):
                if exists[0, w, b, i]:
                    r = OR.add_sub(r, cfg.k0, OW.fastslow_band(params[0, w, b, i], NB), +1, FRAC)
        resid[w] = r
    return resid


def _place(cfg, th):
    k_start, a, e = OW.fastslow_band(th, NB)
    w = np.zeros((2, cfg.n_bins), complex)
    off = k_start - cfg.k0
    w[0, off:off + NB] = a
    w[1, off:off + NB] = e
    return w


def key64(cfg):
    return int(cfg.key[0]) | (int(cfg.key[1]) << 32)


def copy_state(state):
    return {k: v.copy() for k, v in state.items()}
