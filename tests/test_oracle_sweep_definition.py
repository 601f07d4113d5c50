"""The oracle sweep held to the definitions, record by record.

Every decision of ``oracle.mcmc.sweep`` (in-model moves and the flip-all reversible jump of
Alg. 1 / App. C, the ensemble-permuted tempering swaps of Alg. 2 with Eq. temp-final) is
recomputed here from Eq. like alone: the residual of chain (t, w) on band b is built from
scratch as the data minus the cold chain's sources of every other band (as they stood when
the half sweep opened, Sec. V.D) minus the chain's own band-b sources, over the whole data
grid, and the log-likelihood is ``oracle.likelihood.loglike`` of it with walker w's PSD.

* in-model / birth / death: Delta lnL = lnL(after) - lnL(before), and log alpha adds
  beta times it to the prior (or occupancy) term;
* swap between rung t (walker i) and rung t - 1 (walker j): Eq. temp-final,
  beta_t [lnL_i(set of j) - lnL_i(own set)] + beta_{t-1} [lnL_j(set of i) - lnL_j(own set)];
* after every sweep each cold residual equals the data minus the cold chain's templates, bit
  for bit in fixed point.

Three plausible mistakes, planted in the oracle on the CPU, must each fail: swapped
cross-likelihood arguments in the swap, a hotter chain's r' that keeps its own sources, and a
rung-1 swap that updates the wrong walker's cold residual.
"""
import math

import numpy as np
import pytest

from oracle import likelihood as LK
from oracle import mcmc as OM
from oracle import residual as OR
from oracle import waveform as OW

from _sweep_setup import FRAC, NB, cold_residual, copy_state, small_ensemble

BETAS = (1.0, 0.62, 0.41, 0.27)   # four rungs, every beta > 0


def _ensemble():
    cfg, state, dfix, s = small_ensemble(seed=21, n_temps=4, n_walkers=3, n_bands=4, n_max=4, n_per_band=2,
                                         betas=BETAS)
    # a PSD of its own per walker, so that a likelihood taken with the wrong walker's noise
    # differs from the right one
    cfg.psd = np.stack([s * (1.0 + 0.35 * w) for w in range(cfg.n_walkers)])
    return cfg, state, dfix


class _Template:
    """h(theta) on the whole data grid, memoised by parameter values."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.memo = {}

    def __call__(self, th):
        key = tuple(float(x) for x in th)
        h = self.memo.get(key)
        if h is None:
            k_start, a, e = OW.fastslow_band(np.asarray(th, dtype=np.float64), NB)
            h = np.zeros((2, self.cfg.n_bins), complex)
            off = k_start - self.cfg.k0
            h[0, off:off + NB] = a
            h[1, off:off + NB] = e
            self.memo[key] = h
        return h


def _run(cfg, state, n_sweeps):
    """Run the oracle sweeps; every trace record carries the state just before its move
    (the oracle appends a record before it applies the move)."""
    trace = []
    orig = OM._rec

    def rec(*args):
        r = orig(*args)
        r["pre_params"] = state["params"].copy()
        r["pre_exists"] = state["exists"].copy()
        return r

    resid = []
    OM._rec = rec
    try:
        for k in range(n_sweeps):
            OM.sweep(cfg, state, k, trace)
            resid.append((state["params"].copy(), state["exists"].copy(), state["resid"].copy()))
    finally:
        OM._rec = orig
    return trace, resid


def _mismatches(cfg, dfix, trace, resid_after):
    """Records whose Delta lnL or log alpha differs from the definition, and walkers whose cold
    residual is not the data minus their cold templates."""
    data = OR.from_fixed(dfix, FRAC)
    tmpl = _Template(cfg)
    bad = []
    half_start = None
    prev_parity = None
    counted = {"inmodel": 0, "birth": 0, "death": 0, "swap": 0, "hot": 0, "swap_acc": 0, "cold_swap_acc": 0}
    for r in trace:
        if r["parity"] != prev_parity:   # first record of a half sweep: its state opened the half
            half_start = (r["pre_params"][0].copy(), r["pre_exists"][0].copy())
            prev_parity = r["parity"]
        P0h, E0h = half_start
        b = r["b"]

        def lnl(w, P_set, E_set):
            h = np.zeros((2, cfg.n_bins), complex)
            for bb in range(cfg.n_bands):
                if bb == b:
                    continue
                for s in range(cfg.n_max):
                    if E0h[w, bb, s]:
                        h += tmpl(P0h[w, bb, s])
            for s in range(cfg.n_max):
                if E_set[s]:
                    h += tmpl(P_set[s])
            return LK.loglike(data - h, cfg.psd[w], cfg.df)

        P, E = r["pre_params"], r["pre_exists"]
        t, w, kind = r["t"], r["w"], r["kind"]
        if kind in (0, 1, 2):
            if math.isnan(r["dlogl"]):
                continue   # outside the prior support: no likelihood evaluated
            Pb, Eb = P[t, w, b].copy(), E[t, w, b].copy()
            s = r["slot"]
            if kind == 0:
                Pb[s] = r["params"]
                prior = OM.log_prior_shape(r["params"]) - OM.log_prior_shape(P[t, w, b, s])
                counted["inmodel"] += 1
            elif kind == 1:
                Pb[s], Eb[s] = r["params"], True
                prior = cfg.log_occ_odds
                counted["birth"] += 1
            else:
                Eb[s] = False
                prior = -cfg.log_occ_odds
                counted["death"] += 1
            counted["hot"] += t > 0
            want = lnl(w, Pb, Eb) - lnl(w, P[t, w, b], E[t, w, b])
            if abs(r["dlogl"] - want) > 1e-7 * (1.0 + abs(want)):
                bad.append(("dlogl", kind, t, w, b, r["dlogl"], want))
            la = cfg.betas[b, t] * want + prior
            if abs(r["log_alpha"] - la) > 1e-7 * (1.0 + abs(la)):
                bad.append(("log_alpha", kind, t, w, b, r["log_alpha"], la))
        else:
            wi, wj = w, r["partner"]
            si = (P[t, wi, b], E[t, wi, b])
            sj = (P[t - 1, wj, b], E[t - 1, wj, b])
            want = (cfg.betas[b, t] * (lnl(wi, *sj) - lnl(wi, *si))
                    + cfg.betas[b, t - 1] * (lnl(wj, *si) - lnl(wj, *sj)))
            counted["swap"] += 1
            counted["swap_acc"] += r["accepted"]
            counted["cold_swap_acc"] += r["accepted"] and t == 1
            if abs(r["log_alpha"] - want) > 1e-7 * (1.0 + abs(want)):
                bad.append(("swap", t, wi, wj, b, r["log_alpha"], want))
    for k, (P, E, R) in enumerate(resid_after):
        want = cold_residual(cfg, dfix, P, E)
        for w in range(cfg.n_walkers):
            if not np.array_equal(R[w], want[w]):
                bad.append(("cold residual", k, w))
    return bad, counted


def test_every_sweep_decision_follows_the_definitions():
    cfg, state, dfix = _ensemble()
    trace, resid_after = _run(cfg, copy_state(state), 2)
    bad, counted = _mismatches(cfg, dfix, trace, resid_after)
    assert not bad, bad[:5]
    # the check covered every kind of move, hotter chains, and accepted swaps (which change
    # the residual the later records are checked against)
    assert counted["inmodel"] > 30 and counted["birth"] > 30 and counted["death"] > 30, counted
    assert counted["hot"] > 60 and counted["swap"] >= 2 * 2 * 3 * 3 and counted["cold_swap_acc"] > 0, counted


def _planted(monkeypatch, which):
    if which == "swap arguments":
        orig = OM.temp_final_log_alpha
        monkeypatch.setattr(OM, "temp_final_log_alpha",
                            lambda ll_i_m, ll_j_n, ll_i_n, ll_j_m, b1, b2: orig(ll_j_n, ll_i_m, ll_i_n, ll_j_m, b1, b2))
    elif which == "hot window keeps its own sources":
        orig = OM.band_residual
        monkeypatch.setattr(OM, "band_residual",
                            lambda cfg, st, r_snap, rho, t, w, b:
                            rho.copy() if t > 0 else orig(cfg, st, r_snap, rho, t, w, b))
    else:
        orig = OM.swap_cold_update
        monkeypatch.setattr(OM, "swap_cold_update",
                            lambda cfg, st, w, b, old: orig(cfg, st, (w + 1) % cfg.n_walkers, b, old))


@pytest.mark.parametrize("which", ["swap arguments", "hot window keeps its own sources", "wrong cold walker"])
def test_planted_mistakes_fail_the_definition_check(monkeypatch, which):
    cfg, state, dfix = _ensemble()
    _planted(monkeypatch, which)
    trace, resid_after = _run(cfg, copy_state(state), 2)
    bad, _ = _mismatches(cfg, dfix, trace, resid_after)
    assert bad, which
