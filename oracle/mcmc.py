"""Sampler steps of the GB module, FP64 (test infrastructure).

Follows arXiv:2405.04690:

* Eq. rj-acceptance: alpha_RJ = min[1, L(theta_{k,+1}) p(theta_{+1}) / (L(theta_k) q(theta_{+1}))],
  inverted for a removal; likelihoods tempered as L^beta (App. D).
* Eq. temp-orig and Eq. temp-final (App. D): swap acceptance between two walkers with
  walker-attached residuals.
* Alg. 1 (App. A): per band (t, w, b) form the 3-sub-band residual r', subtract the
  band's sources, run n_prop in-model proposals with accept/reject inside the band,
  and for t = 0 write accepted changes back to the cold-chain residual.
* App. C: reversible jump by the "flip-all" basis over n_max slots in random order,
  each a birth (empty slot) or death (occupied slot) accepted or rejected on its own.
* Alg. 2 (App. E): per band, walkers permuted per temperature; current and swapped
  likelihoods from the top temperature down, swap by Eq. temp-final; a swap that
  changes the cold chain updates its residual.
* Sec. V.D: odd bands first, then even bands; three sub-bands per band window.

Readings where the paper is silent: see ``SweepConfig``.
Random numbers come from Philox4x32-10 at fixed counters (``oracle.philox``).
"""
import math

import numpy as np

from . import likelihood as LK
from . import mdn as MD
from . import philox as PX
from . import residual as RS
from . import waveform as WF
from .constants import GM_SUN_C3

SQRT3 = 1.7320508075688772
TWO_PI = 6.283185307179586
K_CHIRP = 96.0 / 5.0 * math.pi ** (8.0 / 3.0)


# ---------------------------------------------------------------- acceptance rules
def rj_log_alpha(dloglike, beta, log_p_new, log_q_new, birth=True):
    """ln of the Eq. rj-acceptance ratio (tempered); removal is the inverse ratio."""
    if birth:
        return beta * dloglike + log_p_new - log_q_new
    return beta * dloglike - log_p_new + log_q_new


def temp_orig_log_alpha(loglike_n, loglike_m, beta_i, beta_j):
    """ln of Eq. temp-orig: (L_n / L_m)^(beta_j - beta_i)."""
    return (beta_j - beta_i) * (loglike_n - loglike_m)


def temp_final_log_alpha(ll_i_m, ll_j_n, ll_i_n, ll_j_m, beta_I, beta_II):
    """ln of Eq. temp-final: L_{i,m}^bI L_{j,n}^bII / (L_{i,n}^bI L_{j,m}^bII)."""
    return beta_I * (ll_i_m - ll_i_n) + beta_II * (ll_j_n - ll_j_m)


# ---------------------------------------------------------------- configuration
class SweepConfig:
    """Sampler set-up. Readings where the paper is silent:

    * bands of ``nb`` bins starting at bin ``band_k0``; band b owns f0 in
      [band_k0 + b nb, band_k0 + (b+1) nb) / T and its sources may move half a band
      into each neighbour (Sec. V.D); a birth in band b draws f0 uniformly over that
      allowance (so the prior proposal equals the band's prior, p/q = 1);
    * slot occupancy prior: independent, P(occupied) = pi_occ (log odds
      ``log_occ_odds``; 0 reproduces Eq. rj-acceptance with no count prior);
    * priors: ln A uniform on [ln A_min, ln A_max]; chirp mass uniform on
      [mc_min, mc_max] (fdot induced, density ~ fdot^-2/5 f0^-11/5); phi0, psi,
      lambda uniform and periodic; cos iota, sin beta uniform on [-1, 1];
    * in-model move: every coordinate perturbed by sigma_c z_c with z_c the
      Irwin-Hall(4) variable (sum of four uniforms, centred, unit variance), except A,
      which is multiplied by exp(sigma_A z) (a symmetric move in ln A, whose Hastings
      factor cancels the 1/A prior);
    * n_prop = round(props_per_source * g) in-model proposals per band task, g the
      number of sources in the band at the start of the task;
    * learned proposal (optional): ``mdn_raw`` gives the mixture-density outputs [272] of
      every (walker, band), as an array [n_walkers][n_bands][272] or a function
      (w, b, rho) -> [272] of the opened window. Births then draw from the defensive
      mixture eps + (1 - eps) q_MDN in the band's unit coordinates (``oracle.mdn``), and a
      fraction ``mdn_inmodel`` of the in-model moves are independence proposals from it.
      rho does not change during the band's pass (it holds the cold chain's sources
      outside band b and all of b's own), so q is one fixed density for every move of the
      pass and Eq. rj-acceptance uses it as it stands;
    * group stretch (optional, the paper's in-model move): ``group`` from ``build_group`` is
      the stationary group (the cold chain's sources of bands b-1, b, b+1 of every walker,
      sorted by f0); a fraction ``group_frac`` of the in-model moves are stretch moves
      Y = X_j + z (X_k - X_j) (Eq. stretch) with X_j drawn uniformly from the
      ``n_friends`` group members nearest in f0 to X_k, z from g(z) ~ 1/sqrt(z) on
      [1/a, a]; see ``group_stretch``.
    """

    def __init__(self, **kw):
        self.tobs = kw["tobs"]
        self.k0 = kw["k0"]                 # residual window start bin
        self.n_bins = kw["n_bins"]
        self.band_k0 = kw["band_k0"]
        self.nb = kw.get("nb", 256)
        self.n_bands = kw["n_bands"]
        self.n_temps = kw["n_temps"]
        self.n_walkers = kw["n_walkers"]
        self.n_max = kw["n_max"]
        self.frac_bits = kw.get("frac_bits", 98)
        self.betas = np.asarray(kw["betas"], dtype=np.float64)        # [n_bands][n_temps]
        self.psd = np.asarray(kw["psd"], dtype=np.float64)            # [n_walkers][n_bins] PSD values
        self.sigma = np.asarray(kw["sigma"], dtype=np.float64)        # 8 widths (ln A first)
        self.log_occ_odds = kw.get("log_occ_odds", 0.0)
        self.props_per_source = kw.get("props_per_source", 1.0)
        self.key = kw.get("key", (0x1234, 0x5678))
        self.ln_a_min = kw.get("ln_a_min", math.log(1e-23))
        self.ln_a_max = kw.get("ln_a_max", math.log(10 ** -21.5))
        self.mc_min = kw.get("mc_min", 0.3)
        self.mc_max = kw.get("mc_max", 0.8)
        self.f_min = kw.get("f_min", 1e-3)
        self.f_max = kw.get("f_max", 4e-3)
        self.df = 1.0 / self.tobs
        self.mdn_raw = kw.get("mdn_raw", None)
        self.mdn_eps = kw.get("mdn_eps", 0.1)
        self.mdn_inmodel = kw.get("mdn_inmodel", 0.0)
        self.group = kw.get("group", None)
        self.group_frac = kw.get("group_frac", 0.0)
        self.n_friends = kw.get("n_friends", 32)
        self.stretch_a = kw.get("stretch_a", 2.0)

    def band_bins(self, b):
        lo = self.band_k0 + b * self.nb
        return lo, lo + self.nb

    def allowance(self, b):
        lo, hi = self.band_bins(b)
        return max(self.f_min, (lo - self.nb / 2) / self.tobs), min(self.f_max, (hi + self.nb / 2) / self.tobs)

    def window(self, b):
        """Residual window of band b: sub-bands b-1, b, b+1 (local offset into the grid, length)."""
        lo, _ = self.band_bins(b)
        return lo - self.nb - self.k0, 3 * self.nb


def chirp_mass(f0, fdot):
    return (fdot / (K_CHIRP * f0 ** (11.0 / 3.0))) ** 0.6 / GM_SUN_C3


def fdot_from_mc(f0, mc):
    return K_CHIRP * f0 ** (11.0 / 3.0) * (mc * GM_SUN_C3) ** (5.0 / 3.0)


def in_support(cfg, th, b):
    """Prior support of a source of band b: f0 in the band's allowance, A in
    [A_min, A_max], |cos iota|, |sin beta| <= 1, chirp mass in [mc_min, mc_max] (written
    as an fdot interval at the source's f0)."""
    a, f0, fd, _, _, ci, sb, _ = th
    lo, hi = cfg.allowance(b)
    if not (lo <= f0 < hi):
        return False
    if not (math.exp(cfg.ln_a_min) <= a <= math.exp(cfg.ln_a_max)):
        return False
    if not (-1.0 <= ci <= 1.0 and -1.0 <= sb <= 1.0):
        return False
    f113 = f0 ** (11.0 / 3.0)
    c_lo = K_CHIRP * (cfg.mc_min * GM_SUN_C3) ** (5.0 / 3.0)
    c_hi = K_CHIRP * (cfg.mc_max * GM_SUN_C3) ** (5.0 / 3.0)
    return c_lo * f113 <= fd <= c_hi * f113


def log_prior_shape(th):
    """Non-uniform part of the prior in the sampled coordinates: ln p(fdot | f0)."""
    return -0.4 * math.log(th[2]) - 2.2 * math.log(th[1])


def dlog_prior(new, th):
    """ln p(new) - ln p(th) of the non-uniform prior factor, from logs of ratios."""
    return -0.4 * math.log(new[2] / th[2]) - 2.2 * math.log(new[1] / th[1])


def _wrap(x, period):
    if x >= period:
        return x - period
    if x < 0.0:
        return x + period
    return x


def _block_words(key, c0, c1, c2, c3, n_blocks):
    out = []
    for m in range(n_blocks):
        out.extend(PX.philox4x32_10((c0 + m, c1, c2, c3), key))
    return out


def propose_in_model(cfg, th, words):
    """In-model proposal from the 48 words of one proposal (word 0 picks the source)."""
    z = [((PX.u24(words[1 + 4 * c]) + PX.u24(words[2 + 4 * c]) + PX.u24(words[3 + 4 * c])
           + PX.u24(words[4 + 4 * c])) - 2.0) * SQRT3 for c in range(8)]
    s = cfg.sigma
    new = list(th)
    new[0] = th[0] * math.exp(s[0] * z[0])
    new[1] = th[1] + s[1] * z[1]
    new[2] = th[2] + s[2] * z[2]
    new[3] = _wrap(th[3] + s[3] * z[3], TWO_PI)
    new[4] = _wrap(th[4] + s[4] * z[4], math.pi)
    new[5] = th[5] + s[5] * z[5]
    new[6] = th[6] + s[6] * z[6]
    new[7] = _wrap(th[7] + s[7] * z[7], TWO_PI)
    return new


def draw_birth(cfg, b, words):
    """Prior draw of a new source in band b from 8 words (u32 each)."""
    lo, hi = cfg.allowance(b)
    u = [PX.u32(w) for w in words[:8]]
    f0 = lo + (hi - lo) * u[0]
    a = math.exp(cfg.ln_a_min + (cfg.ln_a_max - cfg.ln_a_min) * u[1])
    mc = cfg.mc_min + (cfg.mc_max - cfg.mc_min) * u[2]
    return [a, f0, fdot_from_mc(f0, mc), TWO_PI * u[3], math.pi * u[4], 2.0 * u[5] - 1.0, 2.0 * u[6] - 1.0,
            TWO_PI * u[7]]


def _mdn_row(cfg, w, b, rho):
    if cfg.mdn_raw is None:
        return None
    if callable(cfg.mdn_raw):
        return np.asarray(cfg.mdn_raw(w, b, rho), dtype=np.float64)
    return np.asarray(cfg.mdn_raw[w][b], dtype=np.float64)


def mdn_draw(cfg, raw, b, w_def, w_comp, w_dims):
    """Draw from eps prior + (1 - eps) MDN: the prior branch is ``draw_birth`` on the same 8 words."""
    if PX.u32(w_def) < cfg.mdn_eps:
        return draw_birth(cfg, b, w_dims)
    return MD.from_unit(cfg, b, MD.draw_unit(raw, w_comp, w_dims))


def mdn_log_q(cfg, raw, b, th):
    """ln q of source th of band b under the defensive mixture (unit coordinates, prior density 1)."""
    return MD.log_q_defensive(raw, MD.to_unit(cfg, b, th), cfg.mdn_eps)


# ---------------------------------------------------------------- temperature adaptation
def adapt_ladder(betas, acc, iteration, nu=100.0, t0=1000.0):
    """Vousden, Farr & Mandel (2016) ladder update (the paper adapts every ladder this way,
    App. D): with T_0 = 1 and S_i = ln(T_i - T_{i-1}), S_i += kappa (A_i - A_{i+1}) for the
    finite rungs i = 1 .. N-2 (and N-1 when the top rung is finite, with A_N = 0), where A_i
    is the swap acceptance between rungs i-1 and i and kappa = t0 / (nu (t + t0)); then
    T_i = T_{i-1} + e^{S_i}. An infinite top rung (beta = 0) stays."""
    betas = np.asarray(betas, dtype=np.float64)
    n = len(betas)
    if n < 2:
        return betas.copy()
    top_inf = betas[-1] == 0.0
    last = n - 2 if top_inf else n - 1
    if last < 1:
        return betas.copy()
    temps = 1.0 / betas[:last + 1]
    a = list(acc) + [0.0]
    kappa = t0 / (nu * (iteration + t0))
    out = betas.copy()
    t_prev = 1.0
    for i in range(1, last + 1):
        s = math.log(temps[i] - temps[i - 1]) + kappa * (a[i] - a[i + 1])
        t_prev = t_prev + math.exp(s)
        out[i] = 1.0 / t_prev
    return out


def swap_acceptance(cfg, trace):
    """Per band and rung i, the fraction of walkers whose swap between rungs i-1 and i was
    accepted in a sweep's trace: array [n_bands][n_temps] (column 0 unused)."""
    acc = np.zeros((cfg.n_bands, cfg.n_temps))
    for r in trace:
        if r["kind"] == 3 and r["accepted"]:
            acc[r["b"], r["t"]] += 1.0
    return acc / cfg.n_walkers


# ---------------------------------------------------------------- group stretch
STRETCH_PERIODS = (None, None, None, TWO_PI, math.pi, None, None, TWO_PI)


def build_group(cfg, state):
    """Stationary group of every band: the cold chain's sources of bands b-1, b, b+1 of all
    walkers, sorted by f0; list of (f0 array, params array [G][8])."""
    P, E = state["params"], state["exists"]
    out = []
    for b in range(cfg.n_bands):
        rows = []
        for bb in (b - 1, b, b + 1):
            if 0 <= bb < cfg.n_bands:
                for w in range(cfg.n_walkers):
                    for s in range(cfg.n_max):
                        if E[0, w, bb, s]:
                            rows.append(P[0, w, bb, s])
        gp = np.array(rows, dtype=np.float64).reshape(-1, 8)
        order = np.argsort(gp[:, 1], kind="stable")
        gp = gp[order]
        out.append((gp[:, 1].copy(), gp))
    return out


def friends_start(fs, f, nf):
    """Start of the window of the nf group members nearest in f0 to f (fs sorted; nf <= len)."""
    G = len(fs)
    lo = int(np.searchsorted(fs, f, side="left")) - 1
    hi = lo + 1
    for _ in range(nf):
        if hi >= G or (lo >= 0 and f - fs[lo] <= fs[hi] - f):
            lo -= 1
        else:
            hi += 1
    return lo + 1


def _wrap_sym(d, period):
    if d >= 0.5 * period:
        return d - period
    if d < -0.5 * period:
        return d + period
    return d


def group_stretch(cfg, group_b, th, w_j, w_z):
    """Group stretch (Eq. stretch with a stationary group). Coordinates (ln A, f0, fdot, phi0,
    psi, cos i, sin b, lambda); periodic differences taken in [-P/2, P/2). Returns
    (new parameters, ln z) or (new, None) when the move is not reversible as drawn: the
    auxiliary point X_j is not among the nearest friends of the proposed point, or a
    stretched periodic difference leaves [-P/2, P/2). The proposal probability of j,
    1/n_friends both ways, then cancels, and the acceptance is
    z^(d-1) L'^beta p' / (L^beta p) with d = 8."""
    fs, gp = group_b
    G = len(fs)
    nf = min(cfg.n_friends, G)
    s0 = friends_start(fs, th[1], nf)
    j = s0 + PX.ranged(w_j, nf)
    xj = gp[j]
    a = cfg.stretch_a
    zz = (a - 1.0) * PX.u32(w_z) + 1.0
    z = zz * zz / a   # the square as one rounded product (float ** calls pow, not always exact)
    x = [math.log(th[0])] + list(th[1:])
    y0 = [math.log(xj[0])] + list(xj[1:])
    y = []
    ok = True
    for c in range(8):
        per = STRETCH_PERIODS[c]
        if per is None:
            y.append(y0[c] + z * (x[c] - y0[c]))
        else:
            d = z * _wrap_sym(x[c] - y0[c], per)
            if not (-0.5 * per <= d < 0.5 * per):
                ok = False
            v = y0[c] + d
            y.append(_wrap(v, per))
    new = [math.exp(y[0])] + y[1:]
    if ok:
        s1 = friends_start(fs, new[1], nf)
        ok = s1 <= j < s1 + nf
    return new, (math.log(z) if ok else None)


def _rec(kind, t, w, b, slot, seq, acc, parity, dll, la, th, lu):
    """One trace record (the fields of the GPU trace plus ln u)."""
    return {"kind": kind, "t": t, "w": w, "b": b, "slot": slot, "seq": seq, "accepted": bool(acc),
            "parity": parity, "dlogl": dll, "log_alpha": la, "params": None if th is None else list(th), "lu": lu}


def task_id(cfg, t, w, b):
    return (t * cfg.n_walkers + w) * cfg.n_bands + b


# ---------------------------------------------------------------- band likelihood pieces
def _band_window(cfg, th, b):
    """h(theta) placed on band b's window (complex [2][3 nb])."""
    off, n = cfg.window(b)
    return LK.place(WF.fastslow_band(th, cfg.nb, cfg.tobs), cfg.k0 + off, n)


def _swap_dll(cfg, rwin, psd_w, b, th_new, th_old):
    off, n = cfg.window(b)
    bn = WF.fastslow_band(th_new, cfg.nb, cfg.tobs) if th_new is not None else None
    bo = WF.fastslow_band(th_old, cfg.nb, cfg.tobs) if th_old is not None else None
    return LK.delta_loglike_swap(rwin, psd_w, cfg.df, cfg.k0 + off, bn, bo)


def open_band(cfg, state, r_snap, w, b):
    """rho_{w,b}: cold residual of walker w on band b's window with band b's cold sources added back."""
    off, n = cfg.window(b)
    rho = RS.from_fixed(r_snap[w][:, off:off + n], cfg.frac_bits)
    for s in range(cfg.n_max):
        if state["exists"][0, w, b, s]:
            rho = rho + _band_window(cfg, state["params"][0, w, b, s], b)
    return rho


def band_residual(cfg, state, r_snap, rho, t, w, b):
    """r' of Alg. 1 for band (t, w, b) on the band's window: the cold chain reads its residual
    snapshot (which already lacks its own band-b sources); a hotter chain starts from rho_{w,b}
    (the cold chain's residual with band b's cold sources added back) and subtracts its own
    band-b sources (the cold chain's neighbours, Sec. V.D)."""
    off, n = cfg.window(b)
    if t == 0:
        return RS.from_fixed(r_snap[w][:, off:off + n], cfg.frac_bits)
    rp = rho.copy()
    for s in range(cfg.n_max):
        if state["exists"][t, w, b, s]:
            rp = rp - _band_window(cfg, state["params"][t, w, b, s], b)
    return rp


def band_task(cfg, state, r_snap, rho, t, w, b, parity, sweep, trace):
    """Alg. 1 (in-model) followed by the flip-all RJ pass (App. C) for band (t, w, b)."""
    off, n = cfg.window(b)
    psd_w = cfg.psd[w][off:off + n]
    beta = cfg.betas[b, t]
    P = state["params"]
    E = state["exists"]
    R = state["resid"]
    rp = band_residual(cfg, state, r_snap, rho, t, w, b)
    tid = task_id(cfg, t, w, b)

    def apply(th_new, th_old):
        nonlocal rp
        if th_new is not None:
            rp = rp - _band_window(cfg, th_new, b)
        if th_old is not None:
            rp = rp + _band_window(cfg, th_old, b)
        if t == 0:
            if th_old is not None:
                R[w] = RS.add_sub(R[w], cfg.k0, WF.fastslow_band(th_old, cfg.nb, cfg.tobs), -1, cfg.frac_bits)
            if th_new is not None:
                R[w] = RS.add_sub(R[w], cfg.k0, WF.fastslow_band(th_new, cfg.nb, cfg.tobs), +1, cfg.frac_bits)

    raw = _mdn_row(cfg, w, b, rho)
    existing = [s for s in range(cfg.n_max) if E[t, w, b, s]]
    g = len(existing)
    n_prop = int(round(cfg.props_per_source * g))
    for j in range(n_prop):
        words = _block_words(cfg.key, 12 * j, tid, 0 | (parity << 4), sweep, 12)
        k = existing[PX.ranged(words[0], g)]
        th = list(P[t, w, b, k])
        indep = raw is not None and PX.u32(words[35]) < cfg.mdn_inmodel
        grp = (not indep and cfg.group is not None and len(cfg.group[b][0]) > 0
               and PX.u32(words[46]) < cfg.group_frac)
        lnz = 0.0
        if indep:   # independence proposal from the learned mixture
            new = mdn_draw(cfg, raw, b, words[36], words[37], words[38:46])
        elif grp:   # group stretch: words 1 (friend) and 2 (stretch factor)
            new, lnz = group_stretch(cfg, cfg.group[b], th, words[1], words[2])
        else:
            new = propose_in_model(cfg, th, words)
        lu = math.log(PX.u53(words[33], words[34])) if PX.u53(words[33], words[34]) > 0 else -math.inf
        if (grp and lnz is None) or not in_support(cfg, new, b):
            trace.append(_rec(0, t, w, b, k, j, False, parity, float("nan"), -math.inf, new, lu))
            continue
        dll = _swap_dll(cfg, rp, psd_w, b, new, th)
        if indep:   # unit coordinates: prior density 1, q(theta) / q(theta') is the Hastings factor
            la = beta * dll + mdn_log_q(cfg, raw, b, th) - mdn_log_q(cfg, raw, b, new)
        elif grp:   # stretch Jacobian z^(d-1), d = 8 (ln A, f0, fdot and five more)
            la = beta * dll + dlog_prior(new, th) + 7.0 * lnz
        else:
            la = beta * dll + dlog_prior(new, th)
        acc = lu < la
        trace.append(_rec(0, t, w, b, k, j, acc, parity, dll, la, new, lu))
        if acc:
            P[t, w, b, k] = new
            apply(new, th)
    # flip-all reversible jump
    perm_words = _block_words(cfg.key, 0, tid, 1 | (parity << 4), sweep, (cfg.n_max + 3) // 4)
    order = list(range(cfg.n_max))
    wi = 0
    for i in range(cfg.n_max - 1, 0, -1):
        jx = PX.ranged(perm_words[wi], i + 1)
        wi += 1
        order[i], order[jx] = order[jx], order[i]
    for j, s in enumerate(order):
        words = _block_words(cfg.key, 4 * j, tid, 2 | (parity << 4), sweep, 4)
        u = PX.u53(words[8], words[9])
        lu = math.log(u) if u > 0 else -math.inf
        if E[t, w, b, s]:
            th = list(P[t, w, b, s])
            dll = _swap_dll(cfg, rp, psd_w, b, None, th)
            la = beta * dll - cfg.log_occ_odds
            if raw is not None:
                la += mdn_log_q(cfg, raw, b, th)
            acc = lu < la
            trace.append(_rec(2, t, w, b, s, j, acc, parity, dll, la, th, lu))
            if acc:
                E[t, w, b, s] = False
                apply(None, th)
        else:
            if raw is None:
                new = draw_birth(cfg, b, words)
            else:
                new = mdn_draw(cfg, raw, b, words[10], words[11], words[0:8])
                if not in_support(cfg, new, b):
                    trace.append(_rec(1, t, w, b, s, j, False, parity, float("nan"), -math.inf, new, lu))
                    continue
            dll = _swap_dll(cfg, rp, psd_w, b, new, None)
            la = beta * dll + cfg.log_occ_odds
            if raw is not None:
                la -= mdn_log_q(cfg, raw, b, new)
            acc = lu < la
            trace.append(_rec(1, t, w, b, s, j, acc, parity, dll, la, new, lu))
            if acc:
                E[t, w, b, s] = True
                P[t, w, b, s] = new
                apply(new, None)


def _set_sum(cfg, state, t, w, b):
    off, n = cfg.window(b)
    h = np.zeros((2, n), complex)
    for s in range(cfg.n_max):
        if state["exists"][t, w, b, s]:
            h = h + _band_window(cfg, state["params"][t, w, b, s], b)
    return h


def band_loglike(cfg, rho, psd_w, h):
    """Band-local likelihood -1/2 <rho - H|rho - H> on the window (terms outside it cancel in every ratio)."""
    d = rho - h
    return -0.5 * LK.inner(d, d, psd_w, cfg.df)


def swap_band(cfg, state, rhos, b, parity, sweep, trace):
    """Alg. 2 for band b with ensemble-permuted walkers (Eq. temp-final)."""
    T, W = cfg.n_temps, cfg.n_walkers
    off, n = cfg.window(b)
    perms = []
    for t in range(T):
        words = _block_words(cfg.key, 0, b * T + t, 3 | (parity << 4), sweep, (W + 3) // 4)
        order = list(range(W))
        wi = 0
        for i in range(W - 1, 0, -1):
            jx = PX.ranged(words[wi], i + 1)
            wi += 1
            order[i], order[jx] = order[jx], order[i]
        perms.append(order)
    P, E, R = state["params"], state["exists"], state["resid"]
    for c in range(W):
        ws = [perms[t][c] for t in range(T)]
        for t in range(T - 1, 0, -1):
            wt, wm = ws[t], ws[t - 1]
            h_t = _set_sum(cfg, state, t, wt, b)
            h_m = _set_sum(cfg, state, t - 1, wm, b)
            pt, pm = cfg.psd[wt][off:off + n], cfg.psd[wm][off:off + n]
            l_t_at_m = band_loglike(cfg, rhos[(wt, b)], pt, h_m)
            l_t_at_t = band_loglike(cfg, rhos[(wt, b)], pt, h_t)
            l_m_at_t = band_loglike(cfg, rhos[(wm, b)], pm, h_t)
            l_m_at_m = band_loglike(cfg, rhos[(wm, b)], pm, h_m)
            la = temp_final_log_alpha(l_t_at_m, l_m_at_t, l_t_at_t, l_m_at_m, cfg.betas[b, t], cfg.betas[b, t - 1])
            words = PX.philox4x32_10((t, b * W + c, 4 | (parity << 4), sweep), cfg.key)
            u = PX.u53(words[0], words[1])
            lu = math.log(u) if u > 0 else -math.inf
            acc = lu < la
            rec = _rec(3, t, wt, b, c, t, acc, parity, la, la, None, lu)
            rec["partner"] = wm   # the walker of rung t - 1 in this swap
            trace.append(rec)
            if acc:
                old_cold = [list(P[0, wm, b, s]) for s in range(cfg.n_max) if E[0, wm, b, s]] if t == 1 else None
                pa, ea = P[t, wt, b].copy(), E[t, wt, b].copy()
                P[t, wt, b], E[t, wt, b] = P[t - 1, wm, b].copy(), E[t - 1, wm, b].copy()
                P[t - 1, wm, b], E[t - 1, wm, b] = pa, ea
                if t == 1:
                    swap_cold_update(cfg, state, wm, b, old_cold)


def swap_cold_update(cfg, state, w, b, old_cold):
    """After a rung-1 swap the cold chain of walker w holds a new band-b source set: its
    residual d - H gets the old set's templates back and the new set's subtracted."""
    P, E, R = state["params"], state["exists"], state["resid"]
    for th in old_cold:
        R[w] = RS.add_sub(R[w], cfg.k0, WF.fastslow_band(th, cfg.nb, cfg.tobs), -1, cfg.frac_bits)
    for s in range(cfg.n_max):
        if E[0, w, b, s]:
            R[w] = RS.add_sub(R[w], cfg.k0, WF.fastslow_band(P[0, w, b, s], cfg.nb, cfg.tobs), +1, cfg.frac_bits)


def owner_band(cfg, f0):
    """Sub-band whose own bins hold f0 (Sec. V.D): floor((f0 T - band_k0) / nb)."""
    return math.floor((f0 * cfg.tobs - cfg.band_k0) / cfg.nb)


def transfer_ownership(cfg, state):
    """Band-edge ownership transfer of the cold chain (Sec. V.D): a cold-chain source of band b
    whose f0 now lies in the own bins of a neighbour b' = b -+ 1 moves to a free slot of b'.

    Readings: decided on the state at the call (every move at once); band b' takes its
    candidates from b' - 1 first, then from b' + 1, each in ascending slot order, into its
    free slots in ascending order, and a candidate beyond b''s free slots stays where it is
    ("blocked"). Sources whose owner lies outside [0, n_bands), and the hotter chains, stay.
    The model (the set of sources, the residual) does not change: only which band's slots
    hold a source. Returns (moved, blocked); state is updated in place."""
    P0 = state["params"][0].copy()
    E0 = state["exists"][0].copy()
    moved = blocked = 0
    for w in range(cfg.n_walkers):
        for b in range(cfg.n_bands):
            free = [s for s in range(cfg.n_max) if not E0[w, b, s]]
            cands = []
            for nb_ in (b - 1, b + 1):
                if 0 <= nb_ < cfg.n_bands:
                    cands += [(nb_, s) for s in range(cfg.n_max)
                              if E0[w, nb_, s] and owner_band(cfg, P0[w, nb_, s, 1]) == b]
            for k, (src_b, s) in enumerate(cands):
                if k < len(free):
                    state["params"][0, w, b, free[k]] = P0[w, src_b, s]
                    state["exists"][0, w, b, free[k]] = True
                    state["exists"][0, w, src_b, s] = False
                    moved += 1
                else:
                    blocked += 1
    return moved, blocked


def sweep(cfg, state, sweep_index, trace=None, do_swap=True):
    """One sweep: odd bands, then even bands; each half: open, band tasks (Alg. 1 + RJ), swaps (Alg. 2)."""
    if trace is None:
        trace = []
    for parity in (1, 0):
        bands = [b for b in range(cfg.n_bands) if b % 2 == parity]
        r_snap = state["resid"].copy()
        rhos = {(w, b): open_band(cfg, state, r_snap, w, b) for w in range(cfg.n_walkers) for b in bands}
        for b in bands:
            for t in range(cfg.n_temps):
                for w in range(cfg.n_walkers):
                    band_task(cfg, state, r_snap, rhos[(w, b)], t, w, b, parity, sweep_index, trace)
        if do_swap:
            for b in bands:
                swap_band(cfg, state, rhos, b, parity, sweep_index, trace)
    return trace
