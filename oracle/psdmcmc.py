"""Noise-PSD and Galactic-foreground sampler step, FP64 (test infrastructure).

Follows arXiv:2405.04690 Sec. III (Eq. psd), Sec. III.A (the foreground) and Sec. V.B (the PSD
module): each channel A, E has its own two instrument parameters (sqrt(S_oms), sqrt(S_acc)),
the five foreground parameters (A_fg, alpha, f_k, s1, s2) are shared by both channels, and

    S_ch(f) = S_n(f; sqrt(S_oms,ch), sqrt(S_acc,ch)) + S_fg(f; A_fg, alpha, f_k, s1, s2),
    ln L = -1/2 sum_ch 4 df sum_k |R_ch,k|^2 / S_ch,k - sum_ch sum_k ln S_ch,k   (Eq. like).

The module's sampler (Sec. V.B): a fixed-dimensional ensemble MCMC with the regular stretch
proposal (Eq. stretch) over walkers and tempering between neighbouring temperatures of the
same walker index, which share the residual (so Eq. temp-orig applies and no extra
likelihoods are needed).

Readings (the paper gives the structure only): sampled coordinates v = (ln sqrt(S_oms,A), ln sqrt(S_acc,A),
ln sqrt(S_oms,E), ln sqrt(S_acc,E), ln A_fg, alpha, f_k, s1, s2), uniform prior on a box;
ensemble halves [0, W/2) and [W/2, W) updated in turn, partner drawn from the other half;
z ~ 1/sqrt(z) on [1/a, a], a = 2; acceptance z^(d-1) (L_Y / L_X)^beta, d = 9; swaps from the
top temperature down. Random numbers from Philox4x32-10 at these counters:
stretch of walker k at temperature t in half h of sweep s: (t W + k, h, 5, s) -> words 0
(partner), 1 (z), 2-3 (ln u); swap of walker w between t and t-1: (t, w, 6, s) -> words 0-1.
"""
import math

import numpy as np

from . import likelihood as LK
from . import philox as PX
from . import psd as PS

N_PSD = 9


def channel_psd(f, p):
    """(S_A, S_E) for the 9 parameters p = (oms_A, acc_A, oms_E, acc_E, A_fg, alpha, f_k, s1, s2)."""
    fg = PS.foreground_ae(f, p[4], p[5], p[6], p[7], p[8])
    return PS.psd_ae(f, p[0], p[1]) + fg, PS.psd_ae(f, p[2], p[3]) + fg


def loglike(resid, f, df, p):
    """Eq. like of residual [2][n] (A, E) with the per-channel PSD of p."""
    sa, se = channel_psd(f, p)
    return LK.loglike(resid, np.stack([sa, se]), df)


def to_v(p):
    return np.array([math.log(p[0]), math.log(p[1]), math.log(p[2]), math.log(p[3]), math.log(p[4]),
                     p[5], p[6], p[7], p[8]])


def from_v(v):
    return np.array([math.exp(v[0]), math.exp(v[1]), math.exp(v[2]), math.exp(v[3]), math.exp(v[4]),
                     v[5], v[6], v[7], v[8]])


class PsdConfig:
    def __init__(self, n_temps, n_walkers, lo, hi, betas, key, a=2.0):
        self.n_temps, self.n_walkers = n_temps, n_walkers
        self.lo, self.hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
        self.betas = np.asarray(betas, dtype=np.float64)
        self.key = key
        self.a = a


def sweep(cfg, params, logl, resid, f, df, sweep_index, trace=None):
    """One sweep: stretch moves of half 0 then half 1 at every temperature, then swaps.
    params [T][W][9] and logl [T][W] are updated in place; resid [W][2][n]."""
    T, W = cfg.n_temps, cfg.n_walkers
    half = W // 2
    if trace is None:
        trace = []
    for h in (0, 1):
        new_p, new_l = {}, {}
        for t in range(T):
            for k in range(h * half, (h + 1) * half):
                words = PX.philox4x32_10((t * W + k, h, 5, sweep_index), cfg.key)
                j = (1 - h) * half + PX.ranged(words[0], half)
                u = PX.u32(words[1])
                zz = (cfg.a - 1.0) * u + 1.0
                z = zz * zz / cfg.a   # one rounded product (float ** calls pow, not always exact)
                xk, xj = to_v(params[t, k]), to_v(params[t, j])
                y = xj + z * (xk - xj)
                ul = PX.u53(words[2], words[3])
                lu = math.log(ul) if ul > 0 else -math.inf
                inbox = bool(np.all(y >= cfg.lo) and np.all(y <= cfg.hi))
                if inbox:
                    py = from_v(y)
                    ly = loglike(resid[k], f, df, py)
                    la = cfg.betas[t] * (ly - logl[t, k]) + (N_PSD - 1) * math.log(z)
                    acc = lu < la
                else:
                    py, ly, la, acc = None, float("nan"), -math.inf, False
                trace.append({"kind": 5, "t": t, "w": k, "half": h, "accepted": acc, "log_alpha": la, "lu": lu,
                              "logl": ly})
                if acc:
                    new_p[(t, k)], new_l[(t, k)] = py, ly
        for (t, k), py in new_p.items():   # the half moves together: partners are the other half
            params[t, k] = py
            logl[t, k] = new_l[(t, k)]
    for w in range(W):
        for t in range(T - 1, 0, -1):
            words = PX.philox4x32_10((t, w, 6, sweep_index), cfg.key)
            ul = PX.u53(words[0], words[1])
            lu = math.log(ul) if ul > 0 else -math.inf
            la = (cfg.betas[t - 1] - cfg.betas[t]) * (logl[t, w] - logl[t - 1, w])
            acc = lu < la
            trace.append({"kind": 6, "t": t, "w": w, "half": -1, "accepted": acc, "log_alpha": la, "lu": lu,
                          "logl": float("nan")})
            if acc:
                params[[t, t - 1], w] = params[[t - 1, t], w]
                logl[[t, t - 1], w] = logl[[t - 1, t], w]
    return trace
