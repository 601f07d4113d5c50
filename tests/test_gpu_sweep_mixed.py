"""Mixed-precision sweeps with the benchmarked proposals against the float64 oracle.

The mixed sweep (float32 bulk arithmetic, float64 phases and sums) is run with each proposal
variant the benchmark uses: group stretch moves (App. B, Eq. stretch with a stationary group),
the learned proposal (a mixture-density table for births, deaths and independence in-model
moves, defensive eps < 1) and a Gaussian-mixture table fitted on the GPU by gmm_fit (the
paper's refit / search RJ proposals, Sec. V.E and App. G).

Every record of the first half sweep is replayed through the oracle with the GPU's own
proposed parameters and the GPU's decisions (so the replay follows the GPU's chain): the
oracle's Eq. swapsource Delta lnL of that proposal on the band's r', its log alpha (prior
ratio, occupancy odds, mixture densities or the stretch Jacobian z^7 from the same Philox
words) and its decision ln u < log alpha. Required: |Delta lnL error| < 1e-2 and |log alpha
error| < 1e-2 on every record, and every decision equal unless the oracle's log alpha lies
within 1e-2 of ln u (at most two such records). Until a band task's first decision that
differs from the oracle's own run, the GPU's proposals must also equal the oracle's in the unit
coordinates of the prior box: to 1e-5 for the Gaussian and stretch moves and prior births
(float32 steps added in float64), to 1e-4 for the float32 mixture draws.
"""
import math

import numpy as np
import pytest

from oracle import mcmc as OM
from oracle import mdn as MD
from oracle import philox as PX

from _common import torch_cuda
from _sweep_setup import copy_state, small_ensemble
from test_gpu_sweep import _gpu_sweep, _near_truth_table

pytestmark = pytest.mark.gpu


def _lu(words, i):
    u = PX.u53(words[i], words[i + 1])
    return math.log(u) if u > 0 else -math.inf


def _replay_first_half(cfg, state, gtr, ora_trace, sweep=0, parity=1):
    st = copy_state(state)
    r_snap = st["resid"].copy()
    bands = [b for b in range(cfg.n_bands) if b % 2 == parity]
    rhos = {(w, b): OM.open_band(cfg, st, r_snap, w, b) for w in range(cfg.n_walkers) for b in bands}
    by_task, ora = {}, {}
    for r in gtr:
        if int(r["parity"]) == parity and int(r["kind"]) != 3:
            by_task.setdefault((int(r["t"]), int(r["w"]), int(r["b"])), []).append(r)
    for r in ora_trace:
        if r["parity"] == parity and r["kind"] != 3:
            ora[(r["t"], r["w"], r["b"], r["kind"] != 0, r["seq"])] = r
    out = {"worst_dll": 0.0, "worst_la": 0.0, "near": 0, "bad": [], "n": 0, "acc": 0, "kinds": set()}
    P, E = st["params"], st["exists"]
    for b in bands:
        off, nn = cfg.window(b)
        for t in range(cfg.n_temps):
            beta = cfg.betas[b, t]
            for w in range(cfg.n_walkers):
                psd_w = cfg.psd[w][off:off + nn]
                rp = OM.band_residual(cfg, st, r_snap, rhos[(w, b)], t, w, b)
                raw = OM._mdn_row(cfg, w, b, rhos[(w, b)])
                tid = OM.task_id(cfg, t, w, b)
                same_path = True   # no decision has differed from the oracle's own run yet
                recs = sorted(by_task.get((t, w, b), []), key=lambda r: (int(r["kind"]) != 0, int(r["seq"])))
                for r in recs:
                    kind, j, s = int(r["kind"]), int(r["seq"]), int(r["slot"])
                    new = [float(x) for x in r["params"]]
                    ro = ora.get((t, w, b, kind != 0, j))
                    if kind == 0:
                        words = OM._block_words(cfg.key, 12 * j, tid, 0 | (parity << 4), sweep, 12)
                        lu = _lu(words, 33)
                        old = list(P[t, w, b, s])
                        indep = raw is not None and PX.u32(words[35]) < cfg.mdn_inmodel
                        grp = (not indep and cfg.group is not None and len(cfg.group[b][0]) > 0
                               and PX.u32(words[46]) < cfg.group_frac)
                        out["kinds"].add("indep" if indep else "group" if grp else "gauss")
                    else:
                        words = OM._block_words(cfg.key, 4 * j, tid, 2 | (parity << 4), sweep, 4)
                        lu = _lu(words, 8)
                        old = list(P[t, w, b, s]) if kind == 2 else None
                        out["kinds"].add("birth" if kind == 1 else "death")
                    if same_path and ro is not None and kind in (0, 1):   # the proposal itself
                        # unit coordinates of the prior box: float32 mixture draws to 1e-4, the
                        # other moves (float32 steps added in float64) to 1e-5
                        mix = kind == 1 and raw is not None or (kind == 0 and indep)
                        du = np.abs(np.asarray(MD.to_unit(cfg, b, new)) - np.asarray(MD.to_unit(cfg, b, ro["params"])))
                        if np.max(du) > (1e-4 if mix else 1e-5):
                            out["bad"].append(("proposal", t, w, b, kind, j, float(np.max(du))))
                    if math.isnan(float(r["dlogl"])):   # refused without a likelihood (support)
                        if same_path and ro is not None and not math.isnan(ro["dlogl"]):
                            out["bad"].append(("support", t, w, b, kind, j))
                        continue
                    if kind == 0:
                        dll = OM._swap_dll(cfg, rp, psd_w, b, new, old)
                        if indep:
                            prior = OM.mdn_log_q(cfg, raw, b, old) - OM.mdn_log_q(cfg, raw, b, new)
                        elif grp:
                            a = cfg.stretch_a
                            z = ((a - 1.0) * PX.u32(words[2]) + 1.0) ** 2 / a
                            prior = OM.dlog_prior(new, old) + 7.0 * math.log(z)
                        else:
                            prior = OM.dlog_prior(new, old)
                    elif kind == 1:
                        dll = OM._swap_dll(cfg, rp, psd_w, b, new, None)
                        prior = cfg.log_occ_odds - (OM.mdn_log_q(cfg, raw, b, new) if raw is not None else 0.0)
                    else:
                        dll = OM._swap_dll(cfg, rp, psd_w, b, None, old)
                        prior = -cfg.log_occ_odds + (OM.mdn_log_q(cfg, raw, b, old) if raw is not None else 0.0)
                    la = beta * dll + prior
                    out["n"] += 1
                    out["worst_dll"] = max(out["worst_dll"], abs(float(r["dlogl"]) - dll))
                    out["worst_la"] = max(out["worst_la"], abs(float(r["log_alpha"]) - la))
                    acc = bool(r["accepted"])
                    if acc != (lu < la):
                        if abs(la - lu) < 1e-2:
                            out["near"] += 1
                        else:
                            out["bad"].append(("decision", t, w, b, kind, j, la, lu))
                    if ro is not None and acc != ro["accepted"]:
                        same_path = False
                    if acc:   # follow the GPU's chain
                        out["acc"] += 1
                        if kind in (0, 1):
                            rp = rp - OM._band_window(cfg, new, b)
                            P[t, w, b, s] = new
                        if kind in (0, 2):
                            rp = rp + OM._band_window(cfg, old, b)
                        if kind == 1:
                            E[t, w, b, s] = True
                        if kind == 2:
                            E[t, w, b, s] = False
    return out


def _check(res, kinds):
    assert not res["bad"], res["bad"][:5]
    assert res["worst_dll"] < 1e-2, res["worst_dll"]
    assert res["worst_la"] < 1e-2, res["worst_la"]
    assert res["near"] <= 2, res["near"]
    assert res["n"] > 60 and res["acc"] > 10, (res["n"], res["acc"])
    assert kinds <= res["kinds"], res["kinds"]


def test_mixed_sweep_with_group_stretch_matches_oracle():
    torch = torch_cuda()
    cfg, state, _, _ = small_ensemble(seed=17)
    cfg.group, cfg.group_frac, cfg.n_friends = OM.build_group(cfg, state), 0.6, 4
    cfg.props_per_source = 3.0
    trace = OM.sweep(cfg, copy_state(state), 0)
    _, gtr, _ = _gpu_sweep(torch, cfg, state, "mixed", group=(0.6, 4))
    _check(_replay_first_half(cfg, state, gtr, trace), {"group", "gauss", "birth", "death"})


def test_mixed_sweep_with_learned_proposal_matches_oracle():
    # a mixture table with components on the walkers' sources (accepted births and
    # independence moves) and broad ones; eps 0.2, 35 % independence in-model moves
    torch = torch_cuda()
    cfg, state, _, _ = small_ensemble(seed=13)
    table = _near_truth_table(cfg, state, np.random.default_rng(14))
    cfg.mdn_raw, cfg.mdn_eps, cfg.mdn_inmodel = table, 0.2, 0.35
    cfg.props_per_source = 2.0
    trace = OM.sweep(cfg, copy_state(state), 0)
    prop = dict(raw_table=torch.from_numpy(table.astype(np.float32)).cuda(), eps=0.2, inmodel_frac=0.35)
    _, gtr, _ = _gpu_sweep(torch, cfg, state, "mixed", proposal=prop)
    _check(_replay_first_half(cfg, state, gtr, trace), {"indep", "gauss", "birth", "death"})


def test_mixed_sweep_with_gpu_fitted_mixture_table_matches_oracle():
    # the refit proposal: gmm_fit (mixed) on points scattered around every band's cold
    # sources, its table used by both sides
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    cfg, state, _, _ = small_ensemble(seed=19)
    g = np.random.default_rng(20)
    pts = np.full((cfg.n_bands, 400, 8), np.nan, np.float32)
    for b in range(cfg.n_bands):
        us = [MD.to_unit(cfg, b, state["params"][0, w, b, s]) for w in range(cfg.n_walkers)
              for s in range(cfg.n_max) if state["exists"][0, w, b, s]]
        rows = []
        for i in range(400):
            u = np.asarray(us[i % len(us)])
            rows.append(np.clip(u + g.normal(0, 1, 8) * np.array([0.003, 2e-4, 0.02, 0.01, 0.01, 0.01, 0.003, 0.003]),
                                1e-3, 1 - 1e-3))
        pts[b] = np.asarray(rows, np.float32)
    raw = torch.zeros((1, cfg.n_bands, 272), dtype=torch.float32, device="cuda")
    L.gmm_fit(torch.from_numpy(pts).cuda(), raw, n_iter=30, precision=L.GBK_MIXED)
    torch.cuda.synchronize()
    table = np.repeat(raw.cpu().numpy(), cfg.n_walkers, axis=0).astype(np.float64)
    assert np.all(np.isfinite(table))
    cfg.mdn_raw, cfg.mdn_eps, cfg.mdn_inmodel = table, 0.2, 0.35
    cfg.props_per_source = 2.0
    trace = OM.sweep(cfg, copy_state(state), 0)
    prop = dict(raw_table=torch.from_numpy(table.astype(np.float32)).cuda(), eps=0.2, inmodel_frac=0.35)
    _, gtr, _ = _gpu_sweep(torch, cfg, state, "mixed", proposal=prop)
    _check(_replay_first_half(cfg, state, gtr, trace), {"indep", "gauss", "birth", "death"})


def test_mixed_sweep_repeats_bit_for_bit():
    # band tasks are taken from a counter, so which warp runs which band differs from run to run;
    # every result (parameters, occupancy, fixed-point residuals, move counts, the decision trace)
    # must not: two runs of three mixed sweeps from the same state are identical bit for bit
    torch = torch_cuda()
    cfg, state, _, _ = small_ensemble(seed=23, n_temps=3, n_walkers=3, n_bands=6, n_max=4)
    runs = [_gpu_sweep(torch, cfg, copy_state(state), "mixed", sweeps=3) for _ in range(2)]
    (a, ta, sa), (b, tb, sb) = runs
    for k in ("params", "exists", "resid"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(sa, sb)
    assert len(ta) == len(tb) > 0
    def records(tr):   # the trace as a multiset of raw records (its order follows the warps' task order)
        return sorted(r.tobytes() for r in tr)

    assert records(ta) == records(tb)
