"""Pins of the oracle's per-band search sampler (oracle/search.py): a known tempered target
stays stationary under the stretch moves and swaps, the prior (beta = 0) is uniform on the
unit box, the likelihood is Eq. addsource (+1/2 SNR^2 at an injected source on noise-free
data), and the best-point bookkeeping on a worked example."""
import math

import numpy as np

from oracle import constants as OC
from oracle import likelihood as LK
from oracle import psd as OP
from oracle import residual as RS
from oracle import search as SR
from oracle import waveform as WF


def _cfg(n_bands=1, n_temps=2, n_walkers=16, betas=(1.0, 0.25), key=(7, 9)):
    band_k0 = int(math.floor(2.0e-3 * OC.TOBS))
    k0 = band_k0 - 2 * 256
    n_bins = (n_bands + 4) * 256
    f = (k0 + np.arange(n_bins)) * OC.DF
    return SR.SearchConfig(tobs=OC.TOBS, k0=k0, n_bins=n_bins, band_k0=band_k0, n_bands=n_bands, n_temps=n_temps,
                           n_walkers=n_walkers, betas=np.tile(np.asarray(betas[:n_temps]), (n_bands, 1)),
                           psd=OP.psd_ae(f, OC.SQRT_S_OMS, OC.SQRT_S_ACC), key=key)


def test_tempered_gaussian_target_stays_stationary():
    # target at temperature t: N(0.5, s^2 / beta_t) per coordinate (far from the box edges);
    # ensembles started from exact draws keep that law after 15 sweeps (60 independent
    # ensembles): a wrong Jacobian power, z law or swap rule moves the moments
    s = 0.04
    mu = 0.5

    def fn(b, x):
        return -0.5 * float(np.sum((x - mu) ** 2)) / s ** 2

    g = np.random.default_rng(1)
    finals = {0: [], 1: []}
    for e in range(60):
        cfg = _cfg(key=(11, e))
        u = np.empty((1, 2, 16, 8))
        for t in range(2):
            u[0, t] = mu + s / math.sqrt(cfg.betas[0, t]) * g.standard_normal((16, 8))
        ell = SR.evaluate(cfg, None, u, fn)
        for k in range(15):
            SR.sweep(cfg, None, u, ell, k, fn)
        for t in range(2):
            finals[t].append(u[0, t].copy())
    for t, beta in ((0, 1.0), (1, 0.25)):
        x = np.concatenate(finals[t]).ravel()
        sd = s / math.sqrt(beta)
        assert abs(x.mean() - mu) < 4 * sd / math.sqrt(x.size / 16), (t, x.mean())
        assert abs(x.var() / sd ** 2 - 1) < 0.08, (t, x.var() / sd ** 2)


def test_prior_only_search_is_uniform_on_the_box():
    # beta = 0: every walker's law stays uniform on [0, 1]^8 (final states of 40 independent
    # ensembles started from the prior, 40 sweeps each)
    xs = []
    for e in range(40):
        cfg = _cfg(n_temps=1, n_walkers=16, betas=(0.0,), key=(5, e))
        u = SR.init(cfg, 3)
        ell = np.zeros((1, 1, 16))
        for k in range(40):
            SR.sweep(cfg, None, u, ell, k, lambda b, x: 0.0)
        xs.append(u[0, 0].copy())
    x = np.concatenate(xs)
    assert ((x >= 0) & (x <= 1)).all()
    assert np.abs(x.mean(axis=0) - 0.5).max() < 0.05
    assert np.abs(x.var(axis=0) * 12 - 1).max() < 0.15


def test_search_likelihood_is_eq_addsource():
    # noise-free residual = one source of band 0: at its own coordinates l = +1/2 <h|h>;
    # elsewhere l = <h|h'> - 1/2 <h'|h'>
    cfg = _cfg(n_temps=1)
    u0 = np.array([0.8, 0.37, 0.5, 0.2, 0.3, 0.6, 0.4, 0.7])
    th = SR.from_unit(cfg, 0, u0)
    off, n = cfg.window(0)
    h = LK.place(WF.fastslow_band(th, 256, cfg.tobs), cfg.k0 + off, n)
    R = np.zeros((2, cfg.n_bins), complex)
    R[:, off:off + n] = h
    rw = SR.windows(cfg, RS.to_fixed(R, 98), 98)
    psd = cfg.psd[off:off + n]
    hh = LK.inner(h, h, psd, cfg.df)
    assert hh > 100.0
    assert abs(SR.loglike(cfg, rw[0], 0, u0) - 0.5 * hh) < 1e-8 * hh
    u1 = u0.copy()
    u1[1] += 0.01
    h1 = LK.place(WF.fastslow_band(SR.from_unit(cfg, 0, u1), 256, cfg.tobs), cfg.k0 + off, n)
    want = LK.inner(h, h1, psd, cfg.df) - 0.5 * LK.inner(h1, h1, psd, cfg.df)
    assert abs(SR.loglike(cfg, rw[0], 0, u1) - want) < 1e-8 * hh
    # the own-bin prior box: u1 = 0 and 1 are the band's first and last own bins
    lo, hi = cfg.core(0)
    assert abs(SR.from_unit(cfg, 0, np.zeros(8))[1] * cfg.tobs - cfg.band_k0) < 1e-6
    assert abs((hi - lo) * cfg.tobs - 256) < 1e-6


def test_best_point_bookkeeping():
    u = np.arange(2 * 1 * 3 * 8, dtype=float).reshape(2, 1, 3, 8)
    ell = np.array([[[1.0, 5.0, 5.0]], [[-1.0, -2.0, -3.0]]])
    best = np.array([-np.inf, 0.0])
    bu = np.zeros((2, 8))
    stall = np.array([4, 4])
    SR.best_update(u, ell, best, bu, stall)
    assert best.tolist() == [5.0, 0.0] and stall.tolist() == [0, 5]
    assert np.array_equal(bu[0], u[0, 0, 1]) and np.array_equal(bu[1], np.zeros(8))


def test_search_points_map_to_the_sampler_coordinates():
    # own-bin u1 = 0, 1/2, 1 -> allowance coordinate 1/4, 1/2, 3/4 for an interior band; the
    # parameters are unchanged (same source); low-SNR bands give NaN rows
    from oracle import mdn as MD
    from oracle import mcmc as OM
    cfg = _cfg(n_bands=3)
    g = np.random.default_rng(2)
    for u1, want in ((0.0, 0.25), (0.5, 0.5), (1.0, 0.75)):
        u = g.uniform(0.1, 0.9, 8)
        u[1] = u1
        v = SR.to_sweep_unit(cfg, 1, u, 1e-4, 1e-2)
        assert abs(v[1] - want) < 1e-12 and np.array_equal(np.delete(v, 1), np.delete(u, 1))
    scfg = OM.SweepConfig(tobs=cfg.tobs, k0=cfg.k0, n_bins=cfg.n_bins, band_k0=cfg.band_k0, nb=256, n_bands=3,
                          n_temps=1, n_walkers=1, n_max=1, betas=np.ones((3, 1)), psd=np.ones((1, cfg.n_bins)),
                          sigma=np.ones(8), f_min=1e-4, f_max=1e-2)
    u = g.uniform(0.1, 0.9, 8)
    th = SR.from_unit(cfg, 1, u)
    np.testing.assert_allclose(MD.to_unit(scfg, 1, th), SR.to_sweep_unit(cfg, 1, u, 1e-4, 1e-2), rtol=1e-9, atol=1e-12)
    uu = g.uniform(0, 1, (3, 2, 16, 8))
    x = SR.samples(cfg, uu, np.array([50.0, 10.0, -1.0]), 7.0, 1e-4, 1e-2)
    assert np.isfinite(x[0]).all() and np.isnan(x[1]).all() and np.isnan(x[2]).all()


def test_ball_relaunch_is_a_clipped_normal_around_the_best_point():
    # every walker of a band with a best point: best + sigma z, z ~ N(0, 1) per coordinate
    # (Box-Muller on the Philox words), clipped to the box; bands without one are untouched
    from scipy import stats
    cfg = _cfg(n_bands=3, n_temps=4, n_walkers=32)
    u = SR.init(cfg, 1)
    keep = u.copy()
    best = np.array([1.0, -np.inf, 2.0])
    bu = np.array([[0.5] * 8, [0.1] * 8, [0.02] + [0.5] * 7])
    SR.ball(cfg, u, best, bu, 0.01, 3)
    assert np.array_equal(u[1], keep[1])
    z = (u[0] - 0.5) / 0.01
    assert stats.kstest(z.ravel(), "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.1 and abs(z.std() - 1) < 0.1
    assert (u[2, ..., 0] >= 0).all() and (u[2, ..., 0] == 0).any()     # clipped at the box edge


def test_converged_bands_are_left_as_they_are():
    # App. G: a band whose best point has not improved for n_it,max sweeps has converged. With a
    # flat likelihood (bands 0 and 2) the best point is set by the first sweep and never improves,
    # so those bands converge after stall_limit more sweeps and then stay exactly as they are (no
    # records, no moves, stall count frozen); band 1 (a peaked target) keeps sweeping while its
    # best point improves
    cfg = _cfg(n_bands=3)
    cfg.stall_limit = 2

    def fn(b, x):
        return 0.0 if b != 1 else -0.5 * float(np.sum((x - 0.5) ** 2)) / 0.02 ** 2

    u = SR.init(cfg, 5)
    ell = SR.evaluate(cfg, None, u, fn)
    best, bu, stall = np.full(3, -np.inf), np.zeros((3, 8)), np.zeros(3, dtype=np.int64)
    for k in range(8):
        done = SR.converged(cfg, stall)
        before = (u.copy(), ell.copy(), best.copy(), stall.copy())
        trace = SR.search_sweep(cfg, None, u, ell, k, best, bu, stall, fn=fn)
        for b in done:
            assert np.array_equal(u[b], before[0][b]) and np.array_equal(ell[b], before[1][b])
            assert best[b] == before[2][b] and stall[b] == before[3][b]
            assert not any(r["b"] == b for r in trace)
        for b in set(range(3)) - set(done):
            assert any(r["b"] == b for r in trace)
        if k == 0:
            assert stall.tolist() == [0, 0, 0]
    # flat bands: best at sweep 0, stall 1 after sweep 1, 2 after sweep 2: converged from sweep 3
    assert SR.converged(cfg, stall)[:1] == [0] and 2 in SR.converged(cfg, stall)
    assert stall[0] == 2 and stall[2] == 2


def test_band_offset_shifts_only_the_random_streams():
    # a search among several side by side (band0 = i n_bands) is the same search as bands
    # n_bands .. 2 n_bands - 1 of one search over twice the bands: same geometry, same counters,
    # so the same walkers, likelihoods, decisions and best points; band0 = 0 gives other moves
    nb = 2
    cen = [np.array([0.3, 0.6, 0.5, 0.4, 0.5, 0.55, 0.45, 0.5]) + 0.05 * b for b in range(2 * nb)]

    def g(b, x):
        return -0.5 * float(np.sum((x - cen[b]) ** 2)) / 0.05 ** 2

    wide = _cfg(n_bands=2 * nb, key=(3, 4))
    wide.stall_limit = 2
    sub = _cfg(n_bands=nb, key=(3, 4))
    sub.band_k0 = wide.band_k0 + nb * wide.nb
    sub.k0 = wide.k0
    sub.band0 = nb
    sub.stall_limit = 2
    zero = _cfg(n_bands=nb, key=(3, 4))
    zero.band_k0 = sub.band_k0
    zero.k0 = wide.k0
    u_w, u_s, u_z = SR.init(wide, 5), SR.init(sub, 5), SR.init(zero, 5)
    assert np.array_equal(u_w[nb:], u_s) and not np.array_equal(u_s, u_z)
    l_w = SR.evaluate(wide, None, u_w, g)
    l_s = SR.evaluate(sub, None, u_s, lambda b, x: g(b + nb, x))
    bw = (np.full(2 * nb, -np.inf), np.zeros((2 * nb, 8)), np.zeros(2 * nb, dtype=np.int64))
    bs = (np.full(nb, -np.inf), np.zeros((nb, 8)), np.zeros(nb, dtype=np.int64))
    tw, ts = [], []
    for k in range(6):
        SR.search_sweep(wide, None, u_w, l_w, k, *bw, fn=g, trace=tw)
        SR.search_sweep(sub, None, u_s, l_s, k, *bs, fn=lambda b, x: g(b + nb, x), trace=ts)
    assert np.array_equal(u_w[nb:], u_s) and np.array_equal(l_w[nb:], l_s)
    assert np.array_equal(bw[0][nb:], bs[0]) and np.array_equal(bw[1][nb:], bs[1]) and np.array_equal(bw[2][nb:], bs[2])
    keep = [dict(r, b=r["b"] - nb) for r in tw if r["b"] >= nb]
    assert [(r["kind"], r["b"], r["t"], r["w"], r["accepted"]) for r in keep] == \
        [(r["kind"], r["b"], r["t"], r["w"], r["accepted"]) for r in ts]
    SR.ball(wide, u_w, bw[0], bw[1], 0.01, 9)
    SR.ball(sub, u_s, bs[0], bs[1], 0.01, 9)
    assert np.array_equal(u_w[nb:], u_s)
