"""Per-band search sampler (gb_search_*) against the float64 oracle (oracle/search.py).

Seeded residual (noise + two injected sources per band) of one walker, 3 bands x 2
temperatures x 8 walkers. FP64: the prior draws bit for bit, every walker's likelihood to
1e-8 (relative to the band's loudest), and three sweeps with identical decisions: the final
walkers bit for bit (the stretch arithmetic is the oracle's, step by step), likelihoods to
1e-8, the same numbers of accepted moves and swaps, the same best points. Mixed: likelihoods
of the same walkers within 1e-2 + 1e-6 |l| (float32 waveforms and products, as the sweep's
Delta lnL).
"""
import numpy as np
import pytest

from oracle import search as SR

from _common import torch_cuda
from _sweep_setup import FRAC, NB, small_ensemble

pytestmark = pytest.mark.gpu

KEY = (0x51, 0x7E)
SEED = 4
SNR_MIN, F_MIN, F_MAX = 3.0, 1e-3, 4e-3


def _setup():
    cfg, state, dfix, s = small_ensemble(seed=30, n_temps=1, n_walkers=1, n_bands=3, n_max=2, n_per_band=2,
                                         betas=(1.0,))
    scfg = SR.SearchConfig(tobs=cfg.tobs, k0=cfg.k0, n_bins=cfg.n_bins, band_k0=cfg.band_k0, nb=NB, n_bands=3,
                           n_temps=2, n_walkers=8, betas=np.tile([1.0, 0.3], (3, 1)), psd=s, key=KEY)
    return scfg, dfix


def _gpu(torch, scfg, dfix, precision, n_sweeps, stall_limit=0):
    from paper_2405_04690_gb300 import _lib as L
    from paper_2405_04690_gb300 import synth
    dev = torch.device("cuda")
    ctx = L.Context(scfg.tobs, 15.0, scfg.k0, scfg.n_bins)
    plan = L.SearchPlan(ctx, scfg.n_bands, NB, scfg.band_k0, scfg.n_temps, scfg.n_walkers, precision,
                        stall_limit=stall_limit)
    R = torch.from_numpy(dfix[None].copy()).to(dev).contiguous()
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    PS = L.psd_struct(psdp)
    u = torch.empty((scfg.n_bands, scfg.n_temps, scfg.n_walkers, 8), dtype=torch.float64, device=dev)
    ell = torch.empty((scfg.n_bands, scfg.n_temps, scfg.n_walkers), dtype=torch.float64, device=dev)
    key = KEY[0] | (KEY[1] << 32)
    L.gb_search_init(plan, u, key, SEED)
    L.gb_search_windows(plan, L.residual_struct(R, FRAC), 0)
    L.gb_search_eval(plan, u, ell, PS)
    u0, l0 = u.cpu().numpy(), ell.cpu().numpy()
    betas = torch.from_numpy(np.ascontiguousarray(scfg.betas)).to(dev)
    be = torch.full((scfg.n_bands,), -np.inf, dtype=torch.float64, device=dev)
    bu = torch.zeros((scfg.n_bands, 8), dtype=torch.float64, device=dev)
    stall = torch.zeros(scfg.n_bands, dtype=torch.int32, device=dev)
    stats = torch.zeros((2, 2), dtype=torch.int64, device=dev)
    for k in range(n_sweeps):
        L.gb_search_sweep(plan, u, ell, betas, PS, key, k, best=(be, bu, stall), stats=stats)
    x = torch.full((scfg.n_bands, scfg.n_walkers + 3, 8), 7.0, dtype=torch.float32, device=dev)
    L.gb_search_samples(plan, u, be, SNR_MIN, F_MIN, F_MAX, x, 2)
    L.gbk_sync_status(ctx)
    out = (u0, l0, u.cpu().numpy(), ell.cpu().numpy(), be.cpu().numpy(), bu.cpu().numpy(), stall.cpu().numpy(),
           stats.cpu().numpy(), x.cpu().numpy())
    plan.close()
    ctx.close()
    return out


def test_search_fp64_matches_oracle():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    scfg, dfix = _setup()
    rw = SR.windows(scfg, dfix, FRAC)
    u = SR.init(scfg, SEED)
    u_init = u.copy()
    ell = SR.evaluate(scfg, rw, u)
    l_init = ell.copy()
    best, bu, stall = np.full(3, -np.inf), np.zeros((3, 8)), np.zeros(3, dtype=np.int64)
    trace = []
    for k in range(3):
        SR.sweep(scfg, rw, u, ell, k, trace=trace)
        SR.best_update(u, ell, best, bu, stall)
    u0, l0, ug, lg, bg, bug, sg, st, xg = _gpu(torch, scfg, dfix, L.GBK_FP64, 3)
    assert np.array_equal(u0, u_init)
    scale = np.abs(l_init).max(axis=(1, 2))[:, None, None]
    assert (np.abs(l0 - l_init) <= 1e-8 * scale).all(), np.abs(l0 - l_init).max()
    assert np.array_equal(ug, u)
    assert (np.abs(lg - ell) <= 1e-8 * scale).all()
    n_str = sum(1 for r in trace if r["kind"] == 7)
    n_str_acc = sum(1 for r in trace if r["kind"] == 7 and r["accepted"])
    n_sw = sum(1 for r in trace if r["kind"] == 8)
    n_sw_acc = sum(1 for r in trace if r["kind"] == 8 and r["accepted"])
    assert st.tolist() == [[n_str, n_str_acc], [n_sw, n_sw_acc]]
    assert n_str_acc > 0 and n_sw_acc > 0
    assert np.array_equal(bug, bu) and np.array_equal(sg, stall)
    assert (np.abs(bg - best) <= 1e-8 * scale[:, 0, 0]).all()
    # training points for the mixtures: rows 2 .. 2 + W of every band, the rest untouched
    want = SR.samples(scfg, u, best, SNR_MIN, F_MIN, F_MAX).astype(np.float32)
    assert np.isfinite(want).any() and np.isnan(want).any()
    np.testing.assert_allclose(xg[:, 2:2 + scfg.n_walkers], want, rtol=1e-7, atol=0)
    assert (xg[:, :2] == 7.0).all() and (xg[:, 2 + scfg.n_walkers:] == 7.0).all()


def test_search_mixed_likelihoods():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    scfg, dfix = _setup()
    rw = SR.windows(scfg, dfix, FRAC)
    u0, l0, *_ = _gpu(torch, scfg, dfix, L.GBK_MIXED, 0)
    want = SR.evaluate(scfg, rw, u0)
    assert (np.abs(l0 - want) <= 1e-2 + 1e-6 * np.abs(want)).all(), np.abs(l0 - want).max()


def test_search_ball_relaunch_matches_oracle():
    # three sweeps with best points, a relaunch around them (sigma 0.01), the likelihood pass and
    # two more sweeps: walkers within 1e-12 of the oracle's (the Box-Muller logs and cosines may
    # differ in the last bit), likelihoods to 1e-8, the same accepted counts
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    from paper_2405_04690_gb300 import synth
    scfg, dfix = _setup()
    rw = SR.windows(scfg, dfix, FRAC)
    u = SR.init(scfg, SEED)
    ell = SR.evaluate(scfg, rw, u)
    best, bu, stall = np.full(3, -np.inf), np.zeros((3, 8)), np.zeros(3, dtype=np.int64)
    for k in range(3):
        SR.sweep(scfg, rw, u, ell, k)
        SR.best_update(u, ell, best, bu, stall)
    SR.ball(scfg, u, best, bu, 0.01, 5)
    u_ball = u.copy()
    ell = SR.evaluate(scfg, rw, u)
    trace = []
    for k in range(3, 5):
        SR.sweep(scfg, rw, u, ell, k, trace=trace)
    dev = torch.device("cuda")
    ctx = L.Context(scfg.tobs, 15.0, scfg.k0, scfg.n_bins)
    plan = L.SearchPlan(ctx, scfg.n_bands, NB, scfg.band_k0, scfg.n_temps, scfg.n_walkers, L.GBK_FP64)
    R = torch.from_numpy(dfix[None].copy()).to(dev).contiguous()
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    PS = L.psd_struct(psdp)
    ug = torch.empty((scfg.n_bands, scfg.n_temps, scfg.n_walkers, 8), dtype=torch.float64, device=dev)
    lg = torch.empty((scfg.n_bands, scfg.n_temps, scfg.n_walkers), dtype=torch.float64, device=dev)
    key = KEY[0] | (KEY[1] << 32)
    L.gb_search_init(plan, ug, key, SEED)
    L.gb_search_windows(plan, L.residual_struct(R, FRAC), 0)
    L.gb_search_eval(plan, ug, lg, PS)
    betas = torch.from_numpy(np.ascontiguousarray(scfg.betas)).to(dev)
    be = torch.full((scfg.n_bands,), -np.inf, dtype=torch.float64, device=dev)
    bg = torch.zeros((scfg.n_bands, 8), dtype=torch.float64, device=dev)
    sg = torch.zeros(scfg.n_bands, dtype=torch.int32, device=dev)
    for k in range(3):
        L.gb_search_sweep(plan, ug, lg, betas, PS, key, k, best=(be, bg, sg))
    L.gb_search_ball(plan, ug, be, bg, 0.01, key, 5)
    ub = ug.cpu().numpy()
    L.gb_search_eval(plan, ug, lg, PS)
    stats = torch.zeros((2, 2), dtype=torch.int64, device=dev)
    for k in range(3, 5):
        L.gb_search_sweep(plan, ug, lg, betas, PS, key, k, stats=stats)
    L.gbk_sync_status(ctx)
    assert np.abs(ub - u_ball).max() < 1e-12
    assert np.abs(ug.cpu().numpy() - u).max() < 1e-12
    scale = np.abs(ell).max(axis=(1, 2))[:, None, None]
    assert (np.abs(lg.cpu().numpy() - ell) <= 1e-8 * scale).all()
    n_acc = sum(1 for r in trace if r["kind"] == 7 and r["accepted"])
    assert int(stats[0, 1].item()) == n_acc and n_acc > 0
    plan.close()
    ctx.close()


def test_search_fp64_with_convergence_matches_oracle():
    # App. G's convergence test (n_it,max = 2 here): bands whose best point has not improved for
    # two sweeps are left as they are; over 10 sweeps the bands converge at different sweeps, and
    # walkers, best points, stall counts and move counts equal the oracle's bit for bit
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    scfg, dfix = _setup()
    scfg.stall_limit = 2
    rw = SR.windows(scfg, dfix, FRAC)
    u = SR.init(scfg, SEED)
    ell = SR.evaluate(scfg, rw, u)
    scale = np.abs(ell).max(axis=(1, 2))[:, None, None]
    best, bu, stall = np.full(3, -np.inf), np.zeros((3, 8)), np.zeros(3, dtype=np.int64)
    trace, frozen_at = [], {}
    for k in range(10):
        for b in SR.converged(scfg, stall):
            frozen_at.setdefault(b, k)
        SR.search_sweep(scfg, rw, u, ell, k, best, bu, stall, trace=trace)
    assert len(frozen_at) >= 1, stall
    _, _, ug, lg, bg, bug, sg, st, _ = _gpu(torch, scfg, dfix, L.GBK_FP64, 10, stall_limit=2)
    assert np.array_equal(ug, u)
    assert (np.abs(lg - ell) <= 1e-8 * scale).all()
    assert np.array_equal(bug, bu) and np.array_equal(sg, stall)
    assert (np.abs(bg - best) <= 1e-8 * scale[:, 0, 0]).all()
    n_str = sum(1 for r in trace if r["kind"] == 7)
    n_str_acc = sum(1 for r in trace if r["kind"] == 7 and r["accepted"])
    n_sw = sum(1 for r in trace if r["kind"] == 8)
    n_sw_acc = sum(1 for r in trace if r["kind"] == 8 and r["accepted"])
    assert st.tolist() == [[n_str, n_str_acc], [n_sw, n_sw_acc]]


def test_search_sets_one_per_walker_match_oracle():
    # two searches side by side in one plan (n_sets = 2), set s on walker s's residual and PSD
    # row, with its own ladder and the convergence test: each set equals the oracle's search of
    # that walker with the band index offset by s n_bands in the counters (FP64: walkers, best
    # points and stall counts bit for bit, likelihoods to 1e-8, the training points)
    torch = torch_cuda()
    from oracle import constants as OC
    from oracle import psd as OP
    from paper_2405_04690_gb300 import _lib as L
    from paper_2405_04690_gb300 import synth
    cfg, state, dfix, s0 = small_ensemble(seed=31, n_temps=1, n_walkers=2, n_bands=3, n_max=2, n_per_band=2,
                                          betas=(1.0,))
    resid = state["resid"]                       # the two walkers' cold residuals differ
    rows = np.array([[synth.SQRT_S_OMS, synth.SQRT_S_ACC], [1.15 * synth.SQRT_S_OMS, 0.9 * synth.SQRT_S_ACC]])
    f = (cfg.k0 + np.arange(cfg.n_bins)) * OC.DF
    ladders = [np.tile([1.0, 0.3], (3, 1)), np.tile([1.0, 0.45], (3, 1))]
    n_sweeps, nbd = 6, 3
    want = []
    for st_i in range(2):
        sc = SR.SearchConfig(tobs=cfg.tobs, k0=cfg.k0, n_bins=cfg.n_bins, band_k0=cfg.band_k0, nb=NB, n_bands=nbd,
                             n_temps=2, n_walkers=8, betas=ladders[st_i], psd=OP.psd_ae(f, *rows[st_i]), key=KEY,
                             stall_limit=2, band0=st_i * nbd)
        rw = SR.windows(sc, resid[st_i], FRAC)
        u = SR.init(sc, SEED)
        ell = SR.evaluate(sc, rw, u)
        best, bu, stall = np.full(nbd, -np.inf), np.zeros((nbd, 8)), np.zeros(nbd, dtype=np.int64)
        for k in range(n_sweeps):
            SR.search_sweep(sc, rw, u, ell, k, best, bu, stall)
        want.append((u, ell, best, bu, stall, SR.samples(sc, u, best, SNR_MIN, F_MIN, F_MAX).astype(np.float32)))
    dev = torch.device("cuda")
    ctx = L.Context(cfg.tobs, 15.0, cfg.k0, cfg.n_bins)
    plan = L.SearchPlan(ctx, nbd, NB, cfg.band_k0, 2, 8, L.GBK_FP64, stall_limit=2, n_sets=2)
    R = torch.from_numpy(np.ascontiguousarray(resid)).to(dev)
    PS = L.psd_struct(torch.from_numpy(rows).to(dev))
    u = torch.empty((2, nbd, 2, 8, 8), dtype=torch.float64, device=dev)
    ell = torch.empty((2, nbd, 2, 8), dtype=torch.float64, device=dev)
    key = KEY[0] | (KEY[1] << 32)
    L.gb_search_init(plan, u, key, SEED)
    L.gb_search_windows(plan, L.residual_struct(R, FRAC), 0)
    L.gb_search_eval(plan, u, ell, PS)
    betas = torch.from_numpy(np.ascontiguousarray(np.stack(ladders))).to(dev)
    be = torch.full((2, nbd), -np.inf, dtype=torch.float64, device=dev)
    bu = torch.zeros((2, nbd, 8), dtype=torch.float64, device=dev)
    stall = torch.zeros((2, nbd), dtype=torch.int32, device=dev)
    for k in range(n_sweeps):
        L.gb_search_sweep(plan, u, ell, betas, PS, key, k, best=(be, bu, stall))
    x = torch.full((2, nbd, 8, 8), 7.0, dtype=torch.float32, device=dev)
    L.gb_search_samples(plan, u, be, SNR_MIN, F_MIN, F_MAX, x, 0)
    L.gbk_sync_status(ctx)
    ug, lg, bg, bug, sg, xg = (t.cpu().numpy() for t in (u, ell, be, bu, stall, x))
    for st_i in range(2):
        wu, wl, wb, wbu, ws, wx = want[st_i]
        scale = np.abs(wl).max(axis=(1, 2))[:, None, None]
        assert np.array_equal(ug[st_i], wu), st_i
        assert (np.abs(lg[st_i] - wl) <= 1e-8 * scale).all(), st_i
        assert np.array_equal(bug[st_i], wbu) and np.array_equal(sg[st_i], ws), st_i
        assert (np.abs(bg[st_i] - wb) <= 1e-8 * scale[:, 0, 0]).all(), st_i
        np.testing.assert_allclose(xg[st_i], wx, rtol=1e-7, atol=0)
    assert not np.array_equal(ug[0], ug[1])
    plan.close()
    ctx.close()
