"""Seeded synthetic inputs shared by the GPU path, the tests and the oracle.

This module draws random inputs only; it holds none of the likelihood, waveform or
PSD arithmetic. Callers scale the unit normals it returns by their own noise level.

Recipe (the paper's LDC2A data are not available; these draws stand in for them):

* Source parameters (SoA, float64 [8][n]): f0 uniform in [1, 4] mHz (or log-uniform
  over a wider range), log10 A uniform in [-23, -21.5], fdot from the leading-order GR
  chirp with M_chirp uniform in [0.3, 0.8] M_sun, phi0 and psi uniform in [0, 2 pi)
  and [0, pi), cos(iota) and sin(beta) uniform in [-1, 1], lambda uniform in [0, 2 pi).
* Noise: unit complex normals (Re and Im each N(0, 1)); scaled by sqrt(S_n / (4 df))
  they give Re, Im ~ N(0, S_n / (4 df)), i.e. E<n|n> = 2 per bin and channel.
* Per-walker PSD amplitudes: sqrt(S_oms), sqrt(S_acc) log-uniform over +-0.5 dex about
  (15e-12, 3e-15).
"""
import numpy as np

PARAM_NAMES = ("A", "f0", "fdot", "phi0", "psi", "cos_iota", "sin_beta", "lambda")
N_PARAMS = 8

TOBS = 2 ** 21 * 15.0
GM_SUN_C3 = 4.925490947e-6
SQRT_S_OMS = 15e-12
SQRT_S_ACC = 3e-15


def rng(seed):
    """NumPy PCG64 generator for a seed (seed = workload index + 1000 * replicate)."""
    return np.random.Generator(np.random.PCG64(seed))


def fdot_gr(f0, mchirp_sun):
    """Leading-order GR frequency derivative of a circular binary (input recipe)."""
    mc = mchirp_sun * GM_SUN_C3
    return 96.0 / 5.0 * np.pi ** (8.0 / 3.0) * mc ** (5.0 / 3.0) * f0 ** (11.0 / 3.0)


def draw_sources(g, n, f_lo=1e-3, f_hi=4e-3, log_f=False):
    """Draw n sources; returns float64 [8][n] in PARAM_NAMES order."""
    p = np.empty((N_PARAMS, n), dtype=np.float64)
    if log_f:
        p[1] = np.exp(g.uniform(np.log(f_lo), np.log(f_hi), n))
    else:
        p[1] = g.uniform(f_lo, f_hi, n)
    p[0] = 10.0 ** g.uniform(-23.0, -21.5, n)
    p[2] = fdot_gr(p[1], g.uniform(0.3, 0.8, n))
    p[3] = g.uniform(0.0, 2.0 * np.pi, n)
    p[4] = g.uniform(0.0, np.pi, n)
    p[5] = g.uniform(-1.0, 1.0, n)
    p[6] = g.uniform(-1.0, 1.0, n)
    p[7] = g.uniform(0.0, 2.0 * np.pi, n)
    return p


def proposal_widths(params, tobs=TOBS):
    """Per-parameter widths of the in-model Gaussian perturbation (fixed fractions)."""
    df = 1.0 / tobs
    n = params.shape[1]
    w = np.empty((N_PARAMS, n), dtype=np.float64)
    w[0] = 0.05 * params[0]
    w[1] = 0.1 * df
    w[2] = 0.05 * df / tobs
    w[3] = 0.05
    w[4] = 0.05
    w[5] = 0.02
    w[6] = 0.02
    w[7] = 0.02
    return w


def _reflect_unit(x):
    """Fold values back into [-1, 1] by reflection at the edges."""
    x = np.where(x > 1.0, 2.0 - x, x)
    return np.where(x < -1.0, -2.0 - x, x)


def perturb(g, params, widths):
    """Gaussian in-model perturbation of every parameter (cos/sin kept in [-1, 1])."""
    out = params + widths * g.standard_normal(params.shape)
    out[5] = _reflect_unit(out[5])
    out[6] = _reflect_unit(out[6])
    out[0] = np.abs(out[0])
    return out


def unit_complex_normal(g, shape):
    """Complex array whose real and imaginary parts are independent N(0, 1)."""
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def draw_psd_params(g, n_walkers):
    """Per-walker (sqrt(S_oms), sqrt(S_acc)), log-uniform over +-0.5 dex."""
    out = np.empty((n_walkers, 2), dtype=np.float64)
    out[:, 0] = SQRT_S_OMS * 10.0 ** g.uniform(-0.5, 0.5, n_walkers)
    out[:, 1] = SQRT_S_ACC * 10.0 ** g.uniform(-0.5, 0.5, n_walkers)
    return out


def window_for(f_lo, f_hi, margin_bins, tobs=TOBS):
    """Residual window (k0, n_bins) covering [f_lo, f_hi] plus a margin on each side."""
    k_lo = int(np.floor(f_lo * tobs)) - margin_bins
    k_hi = int(np.floor(f_hi * tobs)) + margin_bins
    return k_lo, k_hi - k_lo
