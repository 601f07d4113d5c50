"""The ensemble sweep at the benchmark's full size and launch configuration (16 temperatures x 32
walkers x 369 sub-bands, 2000 injected sources, mixed precision, one step = sweep + ownership
transfer), checked through properties that hold at any size and on sampled windows against
the float64 oracle.

1. Exact bookkeeping: after two steps, every walker's cold residual equals the data minus the
   walker's final cold sources, rebuilt from scratch with the library's own templates (int64
   fixed point, so bit for bit): no accepted change was lost or applied twice anywhere.
2. Independent waveforms on sampled windows: for 24 random (walker, sub-band) windows, the final
   residual plus the oracle's float64 templates of the walker's final cold sources, minus the
   oracle's templates of the injected sources, gives back the injected noise to the float32
   template error (1e-5 of the summed template norms; the mixed waveform's error is ~4e-7 each).
3. The move statistics add up: every proposal is counted once, acceptances never exceed them.

The refit EM (369 groups, one launch) and the search samplers (369 bands x 4 x 32, one launch
per half sweep) at the bench's sizes are checked on sampled groups and bands against the oracle.
"""
import os
import sys

import numpy as np
import pytest

from oracle import residual as OR
from oracle import waveform as OW

from _common import torch_cuda

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_full_size_sweep_bookkeeping_and_sampled_windows():
    torch = torch_cuda()
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as BN
    from paper_2405_04690_gb300 import _lib as L
    dev = torch.device("cuda")
    ens = BN.build_ensemble(seed=1, n_temps=BN.N_T)
    S = BN.build_device_state(torch, L, dev, ens, L.GBK_MIXED, seed=1)
    P0 = S["P"].clone()
    E0 = S["E"].clone()
    R0 = S["resid"].clone()
    stats = torch.zeros((5, 2), dtype=torch.int64, device=dev)
    xfer = torch.zeros(2, dtype=torch.int32, device=dev)
    for k in range(2):
        L.gb_sweep(S["plan"], S["P"], S["E"], S["betas"], S["R"], S["psd"], 0xF011, k,
                   1 | 2 | 4 | (L.SWEEP_REFRESH if k == 0 else 0), stats=stats)
        L.gbk_sweep_transfer(S["plan"], S["P"], S["E"], xfer)
    L.gbk_sync_status(S["ctx"])
    nw, nb_ = BN.N_W, BN.N_BAND
    # (1) rebuild every walker's residual: data = R0 + initial cold templates; expected = data - final cold
    chk = R0.clone()
    RC = L.residual_struct(chk, BN.FRAC_BITS)

    def move(P, E, sign):
        cold = P[0].reshape(-1, 8)[E[0].reshape(-1).bool()]
        wv = E[0].reshape(nw, -1).bool().nonzero()[:, 0].to(torch.int32)
        L.residual_add_sub(S["ctx"], RC, cold.t().contiguous(), torch.full((cold.shape[0],), nb_, dtype=torch.int32,
                           device=dev), nb_, wv, sign, L.GBK_MIXED)

    move(P0, E0, -1)
    move(S["P"], S["E"], +1)
    L.gbk_sync_status(S["ctx"])
    assert torch.equal(chk, S["resid"]), int((chk != S["resid"]).sum().item())
    # (3) statistics
    st = stats.cpu().numpy()
    assert (st[:4, 1] <= st[:4, 0]).all() and st[:4, 0].sum() > 9e6 and xfer[0].item() > 0
    # (2) sampled windows against the oracle's float64 templates
    g = np.random.default_rng(4)
    P = S["P"].cpu().numpy()
    E = S["E"].cpu().numpy().astype(bool)
    R = S["resid"].cpu().numpy()
    noise = OR.from_fixed(S["noise"].cpu().numpy(), BN.FRAC_BITS)
    truth = ens["truth"]
    tobs, k0 = BN.TOBS, ens["k0"]
    worst = 0.0
    for _ in range(24):
        w = int(g.integers(nw))
        b = int(g.integers(1, ens["n_bands"] - 1))
        lo = ens["band_k0"] + (b - 1) * nb_ - k0
        hi = lo + 3 * nb_
        got = OR.from_fixed(R[w], BN.FRAC_BITS)[:, lo:hi]
        acc = np.zeros((2, hi - lo), complex)
        norm = 0.0
        srcs = [(P[0, w][E[0, w]].reshape(-1, 8), +1.0), (truth.T, -1.0)]
        for arr, sign in srcs:
            for th in arr:
                q = int(np.floor(th[1] * tobs)) - k0
                if q + nb_ // 2 <= lo or q - nb_ // 2 >= hi:
                    continue
                ks, a, e = OW.fastslow_band(th, nb_, tobs)
                o = ks - k0 - lo
                i0, i1 = max(0, o), min(hi - lo, o + nb_)
                acc[0, i0:i1] += sign * a[i0 - o:i1 - o]
                acc[1, i0:i1] += sign * e[i0 - o:i1 - o]
                norm += np.linalg.norm(np.concatenate([a, e]))
        diff = got + acc - noise[:, lo:hi]
        rel = np.linalg.norm(diff) / max(norm, 1e-300)
        worst = max(worst, rel)
    assert worst < 1e-5, worst
    S["plan"].close()
    S["ctx"].close()


def test_full_size_em_fit_sampled_bands():
    # the bench's refit: 369 groups of 6400 rows (~1700 present points, clusters of sources that
    # repeat over sweeps and walkers), 16 components, 50 iterations, one launch; 5 sampled groups
    # against the oracle's EM (FP64 1e-9; mixed: log-likelihood within 1e-3 nats per point)
    torch = torch_cuda()
    from oracle import gmm as GM
    from paper_2405_04690_gb300 import _lib as L
    g = np.random.default_rng(21)
    B, P = 369, 6400
    x = np.full((B, P, 8), np.nan, dtype=np.float32)
    for b in range(B):
        k = int(g.integers(3, 9))
        c = g.uniform(0.1, 0.9, (k, 8))
        idx = g.choice(P, int(g.integers(1400, 2000)), replace=False)
        lab = g.integers(0, k, idx.size)
        x[b, idx] = (c[lab] + 0.003 * g.standard_normal((idx.size, 8))).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    sample = [0, 97, 180, 250, 368]
    want = {b: GM.fit(x[b].astype(np.float64), n_iter=50, cap=L.gmm_max_points()) for b in sample}
    for prec in ("fp64", "mixed"):
        raw = torch.empty((1, B, 272), dtype=torch.float32, device="cuda")
        fit = torch.zeros((B, 16, 17), dtype=torch.float64, device="cuda")
        ll = torch.zeros(B, dtype=torch.float64, device="cuda")
        L.gmm_fit(xt, raw, n_iter=50, precision=L.PRECISION[prec], fit_out=fit, loglike=ll)
        fit, ll = fit.cpu().numpy(), ll.cpu().numpy()
        assert np.isfinite(raw.cpu().numpy()).all()
        for b in sample:
            w, mu, var, hist = want[b]
            n = min(int((~np.isnan(x[b]).any(axis=1)).sum()), L.gmm_max_points())
            if prec == "fp64":
                np.testing.assert_allclose(fit[b, :, 0], w, rtol=1e-9, atol=1e-14)
                np.testing.assert_allclose(fit[b, :, 1:9], mu, rtol=1e-9, atol=1e-12)
                np.testing.assert_allclose(fit[b, :, 9:], var, rtol=1e-9, atol=1e-15)
            assert abs(ll[b] - hist[-1]) < (1e-9 * abs(hist[-1]) if prec == "fp64" else 1e-3 * n), (prec, b)


def test_full_size_search_sampled_bands():
    # the bench's search samplers: 369 bands x 4 temperatures x 32 walkers in one launch per
    # half sweep; three sampled bands (each with an injected source) follow the oracle's FP64
    # sampler bit for bit over two sweeps (the bands are independent)
    torch = torch_cuda()
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as BN
    from oracle import constants as OC
    from oracle import psd as OP
    from oracle import search as SR
    from paper_2405_04690_gb300 import _lib as L
    from paper_2405_04690_gb300 import synth
    nb_, B, T, W = BN.N_BAND, 369, 4, 32
    band_k0 = int(np.floor(BN.F_LO * BN.TOBS))
    k0 = band_k0 - 2 * nb_
    n_bins = (B + 4) * nb_
    f = (k0 + np.arange(n_bins)) * OC.DF
    s = OP.psd_ae(f, OC.SQRT_S_OMS, OC.SQRT_S_ACC)
    g = synth.rng(33)
    data = synth.unit_complex_normal(g, (2, n_bins)) * np.sqrt(s / (4 * OC.DF))
    sample = [5, 200, 363]
    for b in sample:
        lo = band_k0 + b * nb_
        th = synth.draw_sources(g, 1, (lo + 20) / OC.TOBS, (lo + nb_ - 20) / OC.TOBS)[:, 0]
        th[0] = 2e-22
        ks, a, e = OW.fastslow_band(th, nb_, OC.TOBS)
        data[0, ks - k0:ks - k0 + nb_] += a
        data[1, ks - k0:ks - k0 + nb_] += e
    rfix = OR.to_fixed(data, BN.FRAC_BITS)
    betas = np.tile([0.5 ** t for t in range(T)], (B, 1))
    cfg = SR.SearchConfig(tobs=OC.TOBS, k0=k0, n_bins=n_bins, band_k0=band_k0, nb=nb_, n_bands=B, n_temps=T,
                          n_walkers=W, betas=betas, psd=s, key=(0x77, 0x12))
    rw = SR.windows(cfg, rfix, BN.FRAC_BITS)
    u = SR.init(cfg, 2)
    ell = SR.evaluate(cfg, rw, u, bands=sample)
    for k in range(2):
        SR.sweep(cfg, rw, u, ell, k, bands=sample)
    dev = torch.device("cuda")
    ctx = L.Context(OC.TOBS, OC.DT, k0, n_bins)
    plan = L.SearchPlan(ctx, B, nb_, band_k0, T, W, L.GBK_FP64)
    ug = torch.empty((B, T, W, 8), dtype=torch.float64, device=dev)
    lg = torch.empty((B, T, W), dtype=torch.float64, device=dev)
    key = 0x77 | (0x12 << 32)
    PS = L.psd_struct(torch.tensor([[OC.SQRT_S_OMS, OC.SQRT_S_ACC]], dtype=torch.float64, device=dev))
    L.gb_search_init(plan, ug, key, 2)
    L.gb_search_windows(plan, L.residual_struct(torch.from_numpy(rfix[None].copy()).to(dev), BN.FRAC_BITS), 0)
    L.gb_search_eval(plan, ug, lg, PS)
    bt = torch.from_numpy(betas).to(dev)
    for k in range(2):
        L.gb_search_sweep(plan, ug, lg, bt, PS, key, k)
    L.gbk_sync_status(ctx)
    ug, lg = ug.cpu().numpy(), lg.cpu().numpy()
    for b in sample:
        assert np.array_equal(ug[b], u[b]), b
        scale = np.abs(ell[b]).max()
        assert (np.abs(lg[b] - ell[b]) <= 1e-8 * scale).all(), b
    plan.close()
    ctx.close()
