"""GPU ensemble sweep (Alg. 1 in-model, flip-all RJ, Alg. 2 tempering) against the oracle.

FP64 sweep: every proposal's Delta lnL within 1e-7, every decision identical, final
parameters and occupancy identical. Mixed sweep: Delta lnL within 1e-2 per proposal up
to the first decision that differs, which must sit within 1e-2 of its threshold.
Plus the exact cold-chain residual bookkeeping and a prior-only statistical check.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import mcmc as OM
from paper_2405_04690_gb300 import synth

from _common import torch_cuda
from _sweep_setup import FRAC, NB, cold_residual, copy_state, key64, small_ensemble

pytestmark = pytest.mark.gpu

ALL = 1 | 2 | 4


def _gpu_sweep(torch, cfg, state, precision, sweeps=1, flags=ALL, trace_cap=20000, proposal=None, group=None):
    from paper_2405_04690_gb300 import _lib as L
    dev = torch.device("cuda")
    ctx = L.Context(cfg.tobs, 15.0, cfg.k0, cfg.n_bins)
    plan = L.SweepPlan(ctx, cfg.n_temps, cfg.n_walkers, cfg.n_bands, cfg.n_max, NB, cfg.band_k0, cfg.sigma,
                       L.PRECISION[precision], log_occ_odds=cfg.log_occ_odds, f_min=cfg.f_min, f_max=cfg.f_max,
                       props_per_source=cfg.props_per_source)
    P = torch.from_numpy(state["params"].copy()).to(dev)
    E = torch.from_numpy(state["exists"].astype(np.uint8)).to(dev)
    R = torch.from_numpy(state["resid"].copy()).to(dev)
    betas = torch.from_numpy(np.ascontiguousarray(cfg.betas)).to(dev)
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    rec = torch.zeros(trace_cap * ctypes.sizeof(L.GbkTraceRec), dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    stats = torch.zeros((5, 2), dtype=torch.int64, device=dev)
    if proposal is not None:
        L.gbk_sweep_set_proposal(plan, **proposal)
        flags |= L.SWEEP_MDN
    if group is not None:   # (fraction, friends): stationary group from the initial state
        L.gbk_sweep_update_group(plan, P, E, group[0], group[1])
    for k in range(sweeps):
        L.gb_sweep(plan, P, E, betas, L.residual_struct(R, FRAC), L.psd_struct(psdp), key64(cfg), k,
                   flags | (L.SWEEP_REFRESH if k == 0 else 0), trace=(rec, trace_cap, cnt), stats=stats)
    L.gbk_sync_status(ctx)
    n = int(cnt.item())
    assert n <= trace_cap
    tr = np.frombuffer(rec.cpu().numpy().tobytes(), dtype=np.dtype(L.TRACE_DTYPE_FIELDS))[:n]
    out = {"params": P.cpu().numpy(), "exists": E.cpu().numpy().astype(bool), "resid": R.cpu().numpy()}
    res = (out, tr, stats.cpu().numpy())
    plan.close()
    ctx.close()
    return res


def _key(r):
    return (int(r["parity"]), int(r["kind"]) if int(r["kind"]) in (0, 3) else 1, int(r["t"]), int(r["w"]),
            int(r["b"]), int(r["slot"]) if int(r["kind"]) == 3 else 0, int(r["seq"]))


def _index(gpu_tr, ora_tr):
    g = {}
    for r in gpu_tr:
        g[_key(r)] = r
    o = {}
    for r in ora_tr:
        kr = (r["parity"], r["kind"] if r["kind"] in (0, 3) else 1, r["t"], r["w"], r["b"],
              r["slot"] if r["kind"] == 3 else 0, r["seq"])
        o[kr] = r
    return g, o


def test_sweep_fp64_matches_oracle_exactly():
    torch = torch_cuda()
    cfg, state, _, _ = small_ensemble(seed=3)
    ora = copy_state(state)
    trace = OM.sweep(cfg, ora, 0)
    out, gtr, stats = _gpu_sweep(torch, cfg, state, "fp64")
    g, o = _index(gtr, trace)
    assert set(g) == set(o), (len(g), len(o))
    worst = 0.0
    for k, ro in o.items():
        rg = g[k]
        assert bool(rg["accepted"]) == ro["accepted"], (k, rg["log_alpha"], ro["log_alpha"], ro["lu"])
        if ro["kind"] != 3:
            assert int(rg["kind"]) == ro["kind"]
            assert int(rg["slot"]) == ro["slot"]
            np.testing.assert_allclose(rg["params"], ro["params"], rtol=1e-13, atol=0)
        if np.isfinite(ro["dlogl"]):
            worst = max(worst, abs(rg["dlogl"] - ro["dlogl"]))
        else:
            assert np.isnan(rg["dlogl"])
    assert worst < 1e-7, worst
    assert np.array_equal(out["exists"], ora["exists"])
    np.testing.assert_allclose(out["params"][ora["exists"]], ora["params"][ora["exists"]], rtol=1e-13, atol=0)
    # residual: same templates, rounded from float64 waveforms that agree to ~1e-13
    diff = np.abs(out["resid"] - ora["resid"]).max()
    assert diff < 2 ** 20, diff
    kinds = stats[:, 0]
    assert kinds[0] > 0 and kinds[1] > 0 and kinds[3] > 0
    assert stats[:4, 0].sum() == len(gtr)


def test_sweep_mixed_matches_oracle_until_a_justified_flip():
    torch = torch_cuda()
    cfg, state, _, _ = small_ensemble(seed=4)
    ora = copy_state(state)
    trace = OM.sweep(cfg, ora, 0)
    out, gtr, _ = _gpu_sweep(torch, cfg, state, "mixed")
    g, o = _index(gtr, trace)
    # band tasks of the first half sweep see identical inputs; compare them in order
    tasks = {}
    for k, ro in o.items():
        if ro["parity"] == 1 and ro["kind"] != 3:
            tasks.setdefault((ro["t"], ro["w"], ro["b"]), []).append((k, ro))
    flips = 0
    worst = 0.0
    for _, recs in tasks.items():
        recs.sort(key=lambda x: (x[1]["kind"] != 0, x[1]["seq"]))
        for k, ro in recs:
            rg = g.get(k)
            assert rg is not None
            if np.isfinite(ro["dlogl"]):
                worst = max(worst, abs(rg["dlogl"] - ro["dlogl"]))
            if bool(rg["accepted"]) != ro["accepted"]:
                assert abs(ro["log_alpha"] - ro["lu"]) < 1e-2
                flips += 1
                break
    assert worst < 1e-2, worst
    assert flips <= 1


def test_sweep_cold_residual_is_exact():
    # The cold-chain residual is changed only by rounded templates, so after several
    # sweeps it equals data - sum(cold templates) bit for bit when the initial model
    # was entered with the same kernels.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    cfg, state, dfix, _ = small_ensemble(seed=5)
    dev = torch.device("cuda")
    ctx = L.Context(cfg.tobs, 15.0, cfg.k0, cfg.n_bins)
    R = torch.from_numpy(np.stack([dfix] * cfg.n_walkers)).to(dev).contiguous()
    RS = L.residual_struct(R, FRAC)

    def move_cold(P, E, sign, prec):
        p = P[0].reshape(-1, 8)[E[0].reshape(-1)]
        wv = np.nonzero(E[0])[0].astype(np.int32)
        if len(wv) == 0:
            return
        pt = torch.from_numpy(np.ascontiguousarray(p.T)).to(dev)
        L.residual_add_sub(ctx, RS, pt, torch.full((len(wv),), NB, dtype=torch.int32, device=dev), NB,
                           torch.from_numpy(wv).to(dev), sign, prec)

    for prec in ("mixed", "fp64"):
        R.copy_(torch.from_numpy(np.stack([dfix] * cfg.n_walkers)))
        move_cold(state["params"], state["exists"], +1, L.PRECISION[prec])
        plan = L.SweepPlan(ctx, cfg.n_temps, cfg.n_walkers, cfg.n_bands, cfg.n_max, NB, cfg.band_k0, cfg.sigma,
                           L.PRECISION[prec], f_min=cfg.f_min, f_max=cfg.f_max)
        P = torch.from_numpy(state["params"].copy()).to(dev)
        E = torch.from_numpy(state["exists"].astype(np.uint8)).to(dev)
        betas = torch.from_numpy(np.ascontiguousarray(cfg.betas)).to(dev)
        psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
        stats = torch.zeros((5, 2), dtype=torch.int64, device=dev)
        for k in range(4):
            L.gb_sweep(plan, P, E, betas, RS, L.psd_struct(psdp), key64(cfg), 10 + k,
                       ALL | (L.SWEEP_REFRESH if k == 0 else 0), stats=stats)
        L.gbk_sync_status(ctx)
        st = stats.cpu().numpy()
        assert st[:, 1].sum() > 0          # something was accepted
        move_cold(P.cpu().numpy(), E.cpu().numpy().astype(bool), -1, L.PRECISION[prec])
        L.gbk_sync_status(ctx)
        assert np.array_equal(R.cpu().numpy(), np.stack([dfix] * cfg.n_walkers)), prec
        plan.close()
    ctx.close()


def test_sweep_prior_only_reproduces_the_prior():
    # beta = 0 everywhere: occupancy of each slot tends to pi = 0.3 (Eq. rj-acceptance
    # with the slot prior odds), and f0 of present sources is uniform over the band's
    # allowance; checked over many sweeps and bands.
    torch = torch_cuda()
    from scipy import stats as sst
    pi = 0.3
    cfg, state, _, _ = small_ensemble(seed=6, n_temps=2, n_walkers=4, n_bands=6, n_max=8, n_per_band=1,
                                      betas=(0.0, 0.0), log_occ_odds=math.log(pi / (1 - pi)))
    from paper_2405_04690_gb300 import _lib as L
    dev = torch.device("cuda")
    ctx = L.Context(cfg.tobs, 15.0, cfg.k0, cfg.n_bins)
    plan = L.SweepPlan(ctx, cfg.n_temps, cfg.n_walkers, cfg.n_bands, cfg.n_max, NB, cfg.band_k0, cfg.sigma,
                       L.GBK_MIXED, log_occ_odds=cfg.log_occ_odds, f_min=cfg.f_min, f_max=cfg.f_max)
    P = torch.from_numpy(state["params"].copy()).to(dev)
    E = torch.from_numpy(state["exists"].astype(np.uint8)).to(dev)
    R = torch.from_numpy(state["resid"].copy()).to(dev)
    betas = torch.zeros((cfg.n_bands, cfg.n_temps), dtype=torch.float64, device=dev)
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    occ, f_rel = [], []
    for k in range(60):
        L.gb_sweep(plan, P, E, betas, L.residual_struct(R, FRAC), L.psd_struct(psdp), 77, k,
                   ALL | (L.SWEEP_REFRESH if k == 0 else 0))
        if k >= 10:
            e = E.cpu().numpy().astype(bool)
            p = P.cpu().numpy()
            occ.append(e.mean())
            for b in range(cfg.n_bands):
                lo, hi = cfg.allowance(b)
                f = p[:, :, b, :, 1][e[:, :, b, :]]
                f_rel.extend(((f - lo) / (hi - lo)).tolist())
    L.gbk_sync_status(ctx)
    occ = float(np.mean(occ))
    n_slots = cfg.n_temps * cfg.n_walkers * cfg.n_bands * cfg.n_max
    assert abs(occ - pi) < 5 * math.sqrt(pi * (1 - pi) / n_slots), occ   # generous: sweeps are correlated
    assert sst.kstest(np.asarray(f_rel[::7]), "uniform").pvalue > 1e-3
    plan.close()
    ctx.close()


def _near_truth_table(cfg, state, g):
    """Mixture tables [W][n_bands][272] whose components sit near the sources of the
    initial state (so learned-proposal births and independence moves are accepted
    sometimes) with broad components mixed in."""
    from oracle import mdn as MD
    from test_oracle_mdn import raw_from
    t = np.empty((cfg.n_walkers, cfg.n_bands, MD.N_OUT))
    for w in range(cfg.n_walkers):
        for b in range(cfg.n_bands):
            us = [MD.to_unit(cfg, b, state["params"][0, w, b, s]) for s in range(cfg.n_max) if state["exists"][0, w, b, s]]
            pi = g.dirichlet(np.ones(MD.N_COMP))
            mu = g.uniform(0.1, 0.9, (MD.N_COMP, MD.N_DIM))
            sd = np.full((MD.N_COMP, MD.N_DIM), 0.3)
            for k, u in enumerate(us[:MD.N_COMP // 2]):
                mu[k] = np.clip(u, 0.02, 0.98)
                sd[k] = [0.002, 1e-4, 0.02, 0.01, 0.01, 0.01, 0.002, 0.002]
            t[w, b] = raw_from(pi, mu, sd)
    return t.astype(np.float32).astype(np.float64)


def test_sweep_fp64_with_learned_proposal_matches_oracle():
    # The same fixed mixture table on both sides: births from the defensive mixture,
    # deaths and a third of the in-model moves with its density; every decision equal.
    torch = torch_cuda()
    cfg, state, _, _ = small_ensemble(seed=13)
    table = _near_truth_table(cfg, state, np.random.default_rng(14))
    cfg.mdn_raw, cfg.mdn_eps, cfg.mdn_inmodel = table, 0.2, 0.35
    ora = copy_state(state)
    trace = OM.sweep(cfg, ora, 0)
    prop = dict(raw_table=torch.from_numpy(table.astype(np.float32)).cuda(), eps=0.2, inmodel_frac=0.35)
    out, gtr, stats = _gpu_sweep(torch, cfg, state, "fp64", proposal=prop)
    g, o = _index(gtr, trace)
    assert set(g) == set(o), (len(g), len(o))
    worst = 0.0
    for k, ro in o.items():
        rg = g[k]
        assert bool(rg["accepted"]) == ro["accepted"], (k, rg["log_alpha"], ro["log_alpha"], ro["lu"])
        if ro["kind"] != 3:
            np.testing.assert_allclose(rg["params"], ro["params"], rtol=1e-12, atol=0)
            if np.isfinite(ro["log_alpha"]):
                assert abs(rg["log_alpha"] - ro["log_alpha"]) < 1e-6 * (1 + abs(ro["log_alpha"]))
        if np.isfinite(ro["dlogl"]):
            worst = max(worst, abs(rg["dlogl"] - ro["dlogl"]))
    assert worst < 1e-7, worst
    assert np.array_equal(out["exists"], ora["exists"])
    # the learned proposal was exercised: accepted births and accepted independence moves
    births = [r for r in trace if r["kind"] == 1 and r["accepted"]]
    assert len(births) > 0 and stats[1, 1] == len(births)


def test_sweep_with_network_equals_sweep_with_its_table():
    # One band (a single half sweep, opened from the initial state): the network run
    # inside gb_sweep on the opened windows gives the same trace, bit for bit, as the
    # table made by mdn_forward on gb_sweep_features of the same state.
    torch = torch_cuda()
    from oracle import mdn as MD
    from paper_2405_04690_gb300 import _lib as L
    cfg, state, _, _ = small_ensemble(seed=15, n_bands=1, n_temps=2, n_walkers=3, n_max=6, betas=(1.0, 0.5))
    dev = torch.device("cuda")
    theta = MD.init_params(np.random.default_rng(16), scale=1.0).astype(np.float32)
    net = L.Mdn(64)
    L.mdn_set_params(net, torch.from_numpy(theta).to(dev))
    # features of the initial state (after a refresh-only sweep that runs no moves)
    ctx = L.Context(cfg.tobs, 15.0, cfg.k0, cfg.n_bins)
    plan = L.SweepPlan(ctx, cfg.n_temps, cfg.n_walkers, cfg.n_bands, cfg.n_max, NB, cfg.band_k0, cfg.sigma,
                       L.GBK_MIXED, f_min=cfg.f_min, f_max=cfg.f_max)
    P = torch.from_numpy(state["params"].copy()).to(dev)
    E = torch.from_numpy(state["exists"].astype(np.uint8)).to(dev)
    R = torch.from_numpy(state["resid"].copy()).to(dev)
    betas = torch.from_numpy(np.ascontiguousarray(cfg.betas)).to(dev)
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    L.gb_sweep(plan, P, E, betas, L.residual_struct(R, FRAC), L.psd_struct(psdp), 1, 0, L.SWEEP_REFRESH)
    x = torch.zeros((cfg.n_walkers, cfg.n_bands, 1024), dtype=torch.bfloat16, device=dev)
    u = torch.zeros((cfg.n_walkers, cfg.n_bands, cfg.n_max, 8), dtype=torch.float32, device=dev)
    L.gb_sweep_features(plan, P, E, L.residual_struct(R, FRAC), L.psd_struct(psdp), x, u)
    raw = torch.zeros((cfg.n_walkers * cfg.n_bands, MD.N_OUT), dtype=torch.float32, device=dev)
    L.mdn_forward(net, x.reshape(-1, 1024), raw)
    torch.cuda.synchronize()
    # features against the oracle's opened window (float32 window, BF16 rounding: 1 ulp)
    xo = np.empty((cfg.n_walkers, 1024))
    for w in range(cfg.n_walkers):
        rho = OM.open_band(cfg, state, state["resid"], w, 0)
        off, n = cfg.window(0)
        xo[w] = MD.features(rho, cfg.psd[w][off:off + n], cfg.df)
    xg = x.float().cpu().numpy()[:, 0, :].astype(np.float64)
    assert np.all(np.abs(xg - xo) <= 2 ** -7 * np.abs(xo) + 1e-3), np.max(np.abs(xg - xo))
    ug = u.cpu().numpy()
    for w in range(cfg.n_walkers):
        for s in range(cfg.n_max):
            if state["exists"][0, w, 0, s]:
                np.testing.assert_allclose(ug[w, 0, s], MD.to_unit(cfg, 0, state["params"][0, w, 0, s]), atol=1e-6)
            else:
                assert np.all(np.isnan(ug[w, 0, s]))
    plan.close()
    ctx.close()
    table = raw.reshape(cfg.n_walkers, cfg.n_bands, MD.N_OUT).contiguous()
    _, t1, s1 = _gpu_sweep(torch, cfg, state, "mixed", proposal=dict(net=net, eps=0.3, inmodel_frac=0.5))
    _, t2, s2 = _gpu_sweep(torch, cfg, state, "mixed", proposal=dict(raw_table=table, eps=0.3, inmodel_frac=0.5))
    assert len(t1) == len(t2) and len(t1) > 0

    def ordered(t):   # records in a fixed order, compared as bytes (NaN-safe, bitwise)
        idx = sorted(range(len(t)), key=lambda i: tuple(int(t[i][f]) for f in ("parity", "kind", "t", "w", "b", "seq",
                                                                                  "slot")))
        return t[idx].tobytes()
    assert ordered(t1) == ordered(t2)
    assert np.array_equal(s1, s2)
    net.close()


def test_sweep_fp64_with_group_stretch_matches_oracle():
    # Both sides build the stationary group from the initial state; 60 % of the in-model
    # moves are group stretches with 4 friends; every decision identical.
    torch = torch_cuda()
    cfg, state, _, _ = small_ensemble(seed=17)
    cfg.group, cfg.group_frac, cfg.n_friends = OM.build_group(cfg, state), 0.6, 4
    cfg.props_per_source = 3.0
    ora = copy_state(state)
    trace = OM.sweep(cfg, ora, 0)
    out, gtr, stats = _gpu_sweep(torch, cfg, state, "fp64", group=(0.6, 4))
    g, o = _index(gtr, trace)
    assert set(g) == set(o), (len(g), len(o))
    worst = 0.0
    for k, ro in o.items():
        rg = g[k]
        assert bool(rg["accepted"]) == ro["accepted"], (k, rg["log_alpha"], ro["log_alpha"], ro["lu"])
        if ro["kind"] != 3:
            np.testing.assert_allclose(rg["params"], ro["params"], rtol=1e-12, atol=1e-300)
            if np.isfinite(ro["log_alpha"]):
                assert abs(rg["log_alpha"] - ro["log_alpha"]) < 1e-6 * (1 + abs(ro["log_alpha"]))
        if np.isfinite(ro["dlogl"]):
            worst = max(worst, abs(rg["dlogl"] - ro["dlogl"]))
    assert worst < 1e-7, worst
    assert np.array_equal(out["exists"], ora["exists"])
    # group moves happened and some were accepted
    moved = [r for r in trace if r["kind"] == 0 and r["accepted"]]
    assert len(moved) > 0


def test_ladder_adaptation_matches_oracle():
    # one FP64 sweep (decisions identical on both sides), then every band's ladder adapted
    # from that sweep's swap acceptance: the oracle's update and the GPU's agree to 1e-12
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    cfg, state, _, _ = small_ensemble(seed=18, n_temps=4, n_walkers=3, betas=(1.0, 0.6, 0.3, 0.0))
    ora = copy_state(state)
    trace = OM.sweep(cfg, ora, 0)
    acc = OM.swap_acceptance(cfg, trace)
    want = np.array([OM.adapt_ladder(cfg.betas[b], acc[b], 7) for b in range(cfg.n_bands)])
    dev = torch.device("cuda")
    ctx = L.Context(cfg.tobs, 15.0, cfg.k0, cfg.n_bins)
    plan = L.SweepPlan(ctx, cfg.n_temps, cfg.n_walkers, cfg.n_bands, cfg.n_max, NB, cfg.band_k0, cfg.sigma,
                       L.GBK_FP64, f_min=cfg.f_min, f_max=cfg.f_max)
    P = torch.from_numpy(state["params"].copy()).to(dev)
    E = torch.from_numpy(state["exists"].astype(np.uint8)).to(dev)
    R = torch.from_numpy(state["resid"].copy()).to(dev)
    betas = torch.from_numpy(np.ascontiguousarray(cfg.betas)).to(dev)
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    L.gb_sweep(plan, P, E, betas, L.residual_struct(R, FRAC), L.psd_struct(psdp), key64(cfg), 0, ALL | L.SWEEP_REFRESH)
    L.gbk_sweep_adapt_temps(plan, betas, 7)
    L.gbk_sync_status(ctx)
    assert np.array_equal(E.cpu().numpy().astype(bool), ora["exists"])
    got = betas.cpu().numpy()
    assert acc[:, 1:].sum() > 0
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
    plan.close()
    ctx.close()


def _edge_state(seed):
    """Small ensemble with cold sources placed in a neighbour's own bins (inside their own
    band's allowance): band 1 -> 2 and band 2 -> 1 of walker 0, band 1 -> 2 of walker 1 into
    a full band 2 (blocked), band 0 below the first band (owner outside: stays), and a hot
    chain's source in a neighbour (hot chains stay)."""
    cfg, state, dfix, _ = small_ensemble(seed=seed, n_temps=3, n_walkers=2, n_bands=4, n_max=4, n_per_band=2)
    P, E = state["params"], state["exists"]

    def at(x):
        return (cfg.band_k0 + x) / cfg.tobs

    P[0, 0, 1, 0, 1] = at(2 * NB + 30)
    P[0, 0, 2, 1, 1] = at(2 * NB - 40)
    P[0, 0, 0, 1, 1] = at(-50)
    P[1, 0, 1, 1, 1] = at(2 * NB + 60)
    for s in (2, 3):                       # walker 1: band 2 full, then band 1 -> 2 is blocked
        P[0, 1, 2, s] = P[0, 1, 2, s - 2]
        P[0, 1, 2, s, 1] = at(2 * NB + 60 + 50 * s)
        P[0, 1, 2, s, 0] *= 0.5
        E[0, 1, 2, s] = True
    P[0, 1, 1, 1, 1] = at(2 * NB + 20)
    state["resid"] = cold_residual(cfg, dfix, P, E)
    return cfg, state


def test_ownership_transfer_matches_oracle_and_keeps_the_caches():
    # FP64: transfer, sweep, transfer, sweep on both sides (the library's caches built first by
    # a refresh-only call). The transfers move the same sources (counts, occupancy and
    # parameters bitwise), and the sweeps after them take identical decisions: the moved
    # templates and the cold template sums the library keeps are those of the new ownership.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    cfg, state = _edge_state(21)
    ora = copy_state(state)
    ora_tr, ora_counts = [], []
    for k in range(2):
        ora_counts.append(OM.transfer_ownership(cfg, ora))
        ora_tr.append(OM.sweep(cfg, ora, k))
    dev = torch.device("cuda")
    ctx = L.Context(cfg.tobs, 15.0, cfg.k0, cfg.n_bins)
    plan = L.SweepPlan(ctx, cfg.n_temps, cfg.n_walkers, cfg.n_bands, cfg.n_max, NB, cfg.band_k0, cfg.sigma,
                       L.GBK_FP64, f_min=cfg.f_min, f_max=cfg.f_max)
    P = torch.from_numpy(state["params"].copy()).to(dev)
    E = torch.from_numpy(state["exists"].astype(np.uint8)).to(dev)
    R = torch.from_numpy(state["resid"].copy()).to(dev)
    betas = torch.from_numpy(np.ascontiguousarray(cfg.betas)).to(dev)
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    cap = 20000
    rec = torch.zeros(cap * ctypes.sizeof(L.GbkTraceRec), dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    counts = torch.zeros(2, dtype=torch.int32, device=dev)
    gpu_counts, bounds = [], [0]
    L.gb_sweep(plan, P, E, betas, L.residual_struct(R, FRAC), L.psd_struct(psdp), key64(cfg), 0, L.SWEEP_REFRESH)
    for k in range(2):
        counts.zero_()
        L.gbk_sweep_transfer(plan, P, E, counts)
        gpu_counts.append(tuple(int(v) for v in counts.cpu().numpy()))
        L.gb_sweep(plan, P, E, betas, L.residual_struct(R, FRAC), L.psd_struct(psdp), key64(cfg), k, ALL,
                   trace=(rec, cap, cnt))
        bounds.append(int(cnt.item()))
    L.gbk_sync_status(ctx)
    assert bounds[-1] <= cap
    tr = np.frombuffer(rec.cpu().numpy().tobytes(), dtype=np.dtype(L.TRACE_DTYPE_FIELDS))[:bounds[-1]]
    assert gpu_counts == ora_counts, (gpu_counts, ora_counts)
    assert ora_counts[0] == (2, 1)
    for k in range(2):
        g, o = _index(tr[bounds[k]:bounds[k + 1]], ora_tr[k])
        assert set(g) == set(o), (k, len(g), len(o))
        for key, ro in o.items():
            assert bool(g[key]["accepted"]) == ro["accepted"], (k, key)
            if np.isfinite(ro["dlogl"]):
                assert abs(g[key]["dlogl"] - ro["dlogl"]) < 1e-7, (k, key)
    assert np.array_equal(E.cpu().numpy().astype(bool), ora["exists"])
    got = P.cpu().numpy()
    np.testing.assert_allclose(got[ora["exists"]], ora["params"][ora["exists"]], rtol=1e-13, atol=0)
    plan.close()
    ctx.close()


def test_unfilled_plan_is_refused_not_run():
    # before the first refresh the plan's caches are empty: a sweep without GBK_SWEEP_REFRESH, a
    # transfer and the feature pass return GBK_EINVAL instead of reading them
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    cfg, state, _, _ = small_ensemble(seed=3)
    dev = torch.device("cuda")
    ctx = L.Context(cfg.tobs, 15.0, cfg.k0, cfg.n_bins)
    plan = L.SweepPlan(ctx, cfg.n_temps, cfg.n_walkers, cfg.n_bands, cfg.n_max, NB, cfg.band_k0, cfg.sigma,
                       L.GBK_MIXED, f_min=cfg.f_min, f_max=cfg.f_max)
    P = torch.from_numpy(state["params"].copy()).to(dev)
    E = torch.from_numpy(state["exists"].astype(np.uint8)).to(dev)
    R = torch.from_numpy(state["resid"].copy()).to(dev)
    betas = torch.from_numpy(np.ascontiguousarray(cfg.betas)).to(dev)
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    RS, PS = L.residual_struct(R, FRAC), L.psd_struct(psdp)
    with pytest.raises(RuntimeError, match="caches are empty"):
        L.gb_sweep(plan, P, E, betas, RS, PS, 1, 0, ALL)
    with pytest.raises(RuntimeError, match="caches are empty"):
        L.gbk_sweep_transfer(plan, P, E)
    u = torch.zeros((cfg.n_walkers, cfg.n_bands, cfg.n_max, 8), dtype=torch.float32, device=dev)
    with pytest.raises(RuntimeError, match="caches are empty"):
        L.gb_sweep_features(plan, P, E, RS, PS, None, u)
    L.gb_sweep(plan, P, E, betas, RS, PS, 1, 0, ALL | L.SWEEP_REFRESH)
    L.gbk_sweep_transfer(plan, P, E)
    L.gbk_sync_status(ctx)
    plan.close()
    ctx.close()
