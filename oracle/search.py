"""Per-band search sampler of the search-RJ proposal, FP64 (test infrastructure).

Sec. V.E and App. G: the "search RJ proposal" runs, independently and simultaneously for every
sub-band, a fixed-dimensional, parallel-tempered ensemble sampler with the stretch proposal
(Eq. stretch) that looks for the highest-likelihood source still left in the residual; the
prior of f0 is narrowed to the sub-band's own bins (no half-band allowance); the best point is
kept, and samples around it are fitted with a Gaussian mixture that becomes the RJ birth
proposal (``oracle.gmm``).

State of band b: T temperatures x W walkers, each one source in the unit coordinates of the
band's prior box (``oracle.mdn.to_unit`` with the own-bin f0 range: u1 = (f0 - lo_b) / (hi_b -
lo_b), lo_b = (band_k0 + b nb) / T, hi_b = lo_b + nb / T). The likelihood of a walker is the
birth Delta lnL of its source against the residual R on the band's three-sub-band window
(Eq. addsource): l(u) = <R|h> - 1/2 <h|h>.

Readings (the paper gives the structure, not the details): stretch moves in the unit box
(the prior is uniform there), ensemble halves [0, W/2) and [W/2, W) updated in turn, partner
from the other half, z ~ 1/sqrt(z) on [1/a, a], a = 2; a proposal outside [0, 1]^8 is
rejected (phases are not wrapped); acceptance z^(d-1) exp(beta (l_Y - l_X)), d = 8; tempering
swaps of each walker index from the top temperature down with Eq. temp-orig. Best point: the
largest l among the cold walkers after each sweep (first walker on ties); a band's search has
converged when that has not improved for n_it,max sweeps. A band qualifies when its best point
has SNR = sqrt(2 l_best) >= the limit (at the amplitude that maximises l, <R|h> = <h|h> and
l = SNR^2 / 2). Random numbers (Philox4x32-10): start of walker (b, t, k) from counters
(b T W + t W + k, m, 9, seed), m = 0, 1 (8 words); stretch of (b, t, k) in half h of search
sweep s: (b T W + t W + k, h, 7, s) -> words 0 (partner), 1 (z), 2-3 (ln u); swap of walker w
between t and t-1: (b W + w, t, 8, s) -> words 0-1. Several searches side by side (the paper
keeps one per walker, each on that walker's residual and PSD) are independent; search number i
of them takes band index band0 + b, band0 = i n_bands, in place of b in these counters so that
their random streams differ.
"""
import math

import numpy as np

from . import likelihood as LK
from . import philox as PX
from . import residual as RS
from . import waveform as WF
from .mcmc import fdot_from_mc

D = 8
TWO_PI = 2.0 * math.pi


class SearchConfig:
    def __init__(self, **kw):
        self.tobs = kw["tobs"]
        self.k0 = kw["k0"]
        self.n_bins = kw["n_bins"]
        self.band_k0 = kw["band_k0"]
        self.nb = kw.get("nb", 256)
        self.n_bands = kw["n_bands"]
        self.n_temps = kw["n_temps"]
        self.n_walkers = kw["n_walkers"]
        self.betas = np.asarray(kw["betas"], dtype=np.float64)     # [n_bands][n_temps]
        self.psd = np.asarray(kw["psd"], dtype=np.float64)         # [n_bins], the residual's walker
        self.key = kw.get("key", (0x1234, 0x5678))
        self.a = kw.get("a", 2.0)
        self.ln_a_min = kw.get("ln_a_min", math.log(1e-23))
        self.ln_a_max = kw.get("ln_a_max", math.log(10 ** -21.5))
        self.mc_min = kw.get("mc_min", 0.3)
        self.mc_max = kw.get("mc_max", 0.8)
        self.df = 1.0 / self.tobs
        # n_it,max (App. G): a band whose best point has not improved for this many sweeps has
        # converged and is left as it is; 0: never
        self.stall_limit = kw.get("stall_limit", 0)
        # offset of the band index in the random-number counters (one search among several)
        self.band0 = kw.get("band0", 0)

    def core(self, b):
        lo = self.band_k0 + b * self.nb
        return lo / self.tobs, (lo + self.nb) / self.tobs

    def window(self, b):
        lo = self.band_k0 + b * self.nb
        return lo - self.nb - self.k0, 3 * self.nb


def from_unit(cfg, b, u):
    """Unit coordinates of band b's own-bin prior box -> source parameters."""
    lo, hi = cfg.core(b)
    f0 = lo + (hi - lo) * u[1]
    mc = cfg.mc_min + (cfg.mc_max - cfg.mc_min) * u[2]
    return [math.exp(cfg.ln_a_min + (cfg.ln_a_max - cfg.ln_a_min) * u[0]), f0, fdot_from_mc(f0, mc),
            TWO_PI * u[3], math.pi * u[4], 2.0 * u[5] - 1.0, 2.0 * u[6] - 1.0, TWO_PI * u[7]]


def windows(cfg, resid_fixed, frac_bits):
    """Complex residual window [2][3 nb] of every band from a fixed-point residual [2][n_bins][2]."""
    out = []
    for b in range(cfg.n_bands):
        off, n = cfg.window(b)
        out.append(RS.from_fixed(resid_fixed[:, off:off + n], frac_bits))
    return out


def loglike(cfg, rwin, b, u):
    """Birth Delta lnL (Eq. addsource) of the source u against band b's residual window."""
    off, n = cfg.window(b)
    band = WF.fastslow_band(from_unit(cfg, b, u), cfg.nb, cfg.tobs)
    return LK.delta_loglike_swap(rwin, cfg.psd[off:off + n], cfg.df, cfg.k0 + off, band, None)


def _ctr(cfg, b, t, k):
    return ((cfg.band0 + b) * cfg.n_temps + t) * cfg.n_walkers + k


def init(cfg, seed):
    """Walkers drawn from the prior: u [B][T][W][8]."""
    u = np.empty((cfg.n_bands, cfg.n_temps, cfg.n_walkers, D))
    for b in range(cfg.n_bands):
        for t in range(cfg.n_temps):
            for k in range(cfg.n_walkers):
                w = list(PX.philox4x32_10((_ctr(cfg, b, t, k), 0, 9, seed), cfg.key)) + \
                    list(PX.philox4x32_10((_ctr(cfg, b, t, k), 1, 9, seed), cfg.key))
                u[b, t, k] = [PX.u32(x) for x in w]
    return u


def ball(cfg, u, best_ell, best_u, sigma, seed):
    """Relaunch around the best points (App. G: a new ball of points around the maximum-likelihood
    point, the search then run again): every walker of a band with a best point becomes
    clip(best + sigma z, 0, 1), z standard normal by Box-Muller on Philox words at counters
    (chain, m, 10, seed), m = 0, 1: z_{2i}, z_{2i+1} = sqrt(-2 ln u_a) (cos, sin)(2 pi u_b) from
    the word pair (2i, 2i+1) of the 8 words. Bands without a best point (best_ell = -inf) keep
    their walkers. u [B][T][W][8] is updated in place."""
    for b in range(cfg.n_bands):
        if not np.isfinite(best_ell[b]):
            continue
        for t in range(cfg.n_temps):
            for k in range(cfg.n_walkers):
                c = _ctr(cfg, b, t, k)
                w = list(PX.philox4x32_10((c, 0, 10, seed), cfg.key)) + list(PX.philox4x32_10((c, 1, 10, seed), cfg.key))
                z = np.empty(D)
                for i in range(D // 2):
                    r = math.sqrt(-2.0 * math.log(PX.u32(w[2 * i])))
                    a = 2.0 * math.pi * PX.u32(w[2 * i + 1])
                    z[2 * i], z[2 * i + 1] = r * math.cos(a), r * math.sin(a)
                u[b, t, k] = np.clip(best_u[b] + sigma * z, 0.0, 1.0)


def evaluate(cfg, rwins, u, fn=None, bands=None):
    """l of every walker: [B][T][W] (only the listed bands when given, zero elsewhere); fn(b, u)
    replaces the likelihood (tests)."""
    f = fn or (lambda b, x: loglike(cfg, rwins[b], b, x))
    out = np.zeros((cfg.n_bands, cfg.n_temps, cfg.n_walkers))
    for b in (range(cfg.n_bands) if bands is None else bands):
        for t in range(cfg.n_temps):
            for k in range(cfg.n_walkers):
                out[b, t, k] = f(b, u[b, t, k])
    return out


def sweep(cfg, rwins, u, ell, s, fn=None, trace=None, bands=None):
    """One search sweep of every band (or of the listed bands: the bands are independent):
    stretch moves of half 0 then half 1 at every temperature, then tempering swaps. u
    [B][T][W][8] and ell [B][T][W] are updated in place."""
    f = fn or (lambda b, x: loglike(cfg, rwins[b], b, x))
    T, W = cfg.n_temps, cfg.n_walkers
    half = W // 2
    if trace is None:
        trace = []
    for b in (range(cfg.n_bands) if bands is None else bands):
        for h in (0, 1):
            for t in range(T):
                for k in range(h * half, (h + 1) * half):
                    words = PX.philox4x32_10((_ctr(cfg, b, t, k), h, 7, s), cfg.key)
                    j = (1 - h) * half + PX.ranged(words[0], half)
                    zz = (cfg.a - 1.0) * PX.u32(words[1]) + 1.0
                    z = zz * zz / cfg.a   # one rounded product (float ** calls pow, not always exact)
                    y = u[b, t, j] + z * (u[b, t, k] - u[b, t, j])
                    ul = PX.u53(words[2], words[3])
                    lu = math.log(ul) if ul > 0 else -math.inf
                    if np.all(y >= 0.0) and np.all(y <= 1.0):
                        ly = f(b, y)
                        la = cfg.betas[b, t] * (ly - ell[b, t, k]) + (D - 1) * math.log(z)
                    else:
                        ly, la = float("nan"), -math.inf
                    acc = lu < la
                    trace.append({"kind": 7, "b": b, "t": t, "w": k, "half": h, "accepted": acc, "ell": ly,
                                  "log_alpha": la})
                    if acc:
                        u[b, t, k] = y
                        ell[b, t, k] = ly
        for w in range(W):
            for t in range(T - 1, 0, -1):
                words = PX.philox4x32_10(((cfg.band0 + b) * W + w, t, 8, s), cfg.key)
                ul = PX.u53(words[0], words[1])
                lu = math.log(ul) if ul > 0 else -math.inf
                la = (cfg.betas[b, t - 1] - cfg.betas[b, t]) * (ell[b, t, w] - ell[b, t - 1, w])
                acc = lu < la
                trace.append({"kind": 8, "b": b, "t": t, "w": w, "half": -1, "accepted": acc, "ell": float("nan"),
                              "log_alpha": la})
                if acc:
                    u[b, [t, t - 1], w] = u[b, [t - 1, t], w]
                    ell[b, [t, t - 1], w] = ell[b, [t - 1, t], w]
    return trace


def best_update(u, ell, best_ell, best_u, stall, bands=None):
    """After a sweep: the largest cold-chain l of every band (or of the listed bands; first walker
    on ties) replaces the band's best point if larger (stall = 0), else stall += 1. Arrays updated
    in place."""
    for b in (range(ell.shape[0]) if bands is None else bands):
        k = int(np.argmax(ell[b, 0]))
        if ell[b, 0, k] > best_ell[b]:
            best_ell[b] = ell[b, 0, k]
            best_u[b] = u[b, 0, k]
            stall[b] = 0
        else:
            stall[b] += 1


def converged(cfg, stall):
    """Bands whose search has converged (App. G): n_it,max = stall_limit sweeps without a better
    best point."""
    return [b for b in range(cfg.n_bands) if cfg.stall_limit > 0 and stall[b] >= cfg.stall_limit]


def search_sweep(cfg, rwins, u, ell, s, best_ell, best_u, stall, fn=None, trace=None):
    """One sweep with the convergence test: the bands that have converged at its start are left as
    they are, the others sweep and update their best points."""
    done = set(converged(cfg, stall))
    active = [b for b in range(cfg.n_bands) if b not in done]
    trace = sweep(cfg, rwins, u, ell, s, fn=fn, trace=trace, bands=active)
    best_update(u, ell, best_ell, best_u, stall, bands=active)
    return trace


def to_sweep_unit(cfg, b, u, f_min, f_max):
    """A search point of band b in the sampler's unit coordinates (``oracle.mdn.to_unit``), whose
    f0 coordinate spans the band's allowance (own bins +- half a band, clipped to [f_min,
    f_max]) instead of its own bins; the other coordinates are the same."""
    lo, hi = cfg.core(b)
    f0 = lo + (hi - lo) * u[1]
    lob = cfg.band_k0 + b * cfg.nb
    alo = max(f_min, (lob - cfg.nb / 2) / cfg.tobs)
    ahi = min(f_max, (lob + cfg.nb + cfg.nb / 2) / cfg.tobs)
    out = np.array(u, dtype=np.float64)
    out[1] = (f0 - alo) / (ahi - alo)
    return out


def samples(cfg, u, best_ell, snr_min, f_min, f_max):
    """Training points of the search-RJ mixtures from one sweep: the cold walkers of every band
    in the sampler's unit coordinates, [B][W][8]; rows of a band whose best point has
    sqrt(2 l_best) < snr_min are NaN (the band gets no fitted component)."""
    out = np.full((cfg.n_bands, cfg.n_walkers, D), np.nan)
    for b in range(cfg.n_bands):
        if best_ell[b] > 0 and math.sqrt(2.0 * best_ell[b]) >= snr_min:
            for k in range(cfg.n_walkers):
                out[b, k] = to_sweep_unit(cfg, b, u[b, 0, k], f_min, f_max)
    return out
