"""Pins of the oracle's sampler pieces: Eq. temp-final vs Eq. temp-orig, the
reversible-jump ratio, the swap rate of a two-temperature Gaussian toy, the Philox
generator's known answers and uniformity, the fdot prior and support induced by a uniform chirp
mass, and a prior-only run of the full sweep."""
import math

import numpy as np
from scipy import integrate, stats

from oracle import mcmc as OM
from oracle import philox as PX

from _sweep_setup import copy_state, small_ensemble


def test_temp_final_reduces_to_temp_orig_for_shared_likelihoods():
    # App. D: with L_{i,n} = L_{j,n} = L_n and L_{i,m} = L_{j,m} = L_m, Eq. temp-final
    # equals Eq. temp-orig.
    g = np.random.default_rng(1)
    for _ in range(100):
        ln, lm = g.normal(0, 50, 2)
        bi, bj = g.uniform(0, 1, 2)
        a2 = OM.temp_final_log_alpha(lm, ln, ln, lm, bi, bj)
        a1 = OM.temp_orig_log_alpha(ln, lm, bi, bj)
        assert abs(a1 - a2) < 1e-10 * (1 + abs(a1))


def test_rj_ratio_is_inverted_for_removal():
    for dll in (-3.0, 0.5, 12.0):
        up = OM.rj_log_alpha(dll, 0.7, -1.2, -2.0, birth=True)
        down = OM.rj_log_alpha(-dll, 0.7, -1.2, -2.0, birth=False)
        assert abs(up + down) < 1e-12


def test_swap_rate_of_two_temperature_gaussian_toy():
    # Two chains at beta = 1 and 0.4 sample N(0, 1/beta) exactly; the mean swap
    # acceptance min(1, exp(alpha)) with ln L = -x^2/2 equals the integral over both
    # stationary densities (a wrong sign in the swap ratio gives a different rate).
    b1, b2 = 1.0, 0.4
    g = np.random.default_rng(2)
    x1 = g.normal(0, 1 / math.sqrt(b1), 400000)
    x2 = g.normal(0, 1 / math.sqrt(b2), 400000)
    l1, l2 = -0.5 * x1 ** 2, -0.5 * x2 ** 2
    la = OM.temp_orig_log_alpha(l2, l1, b1, b2)
    rate = np.mean(np.minimum(1.0, np.exp(la)))

    def dens(y, x):
        a = (b2 - b1) * (-0.5 * y ** 2 + 0.5 * x ** 2)
        return min(1.0, math.exp(a)) * stats.norm.pdf(x, 0, 1 / math.sqrt(b1)) * stats.norm.pdf(y, 0, 1 / math.sqrt(b2))

    want, _ = integrate.dblquad(dens, -8, 8, -12, 12, epsabs=1e-7)
    assert abs(rate - want) < 5e-3, (rate, want)
    # the swap must favour moving the hotter chain's higher-likelihood state down
    assert want < 1.0


def test_philox_words_are_uniform_and_counter_distinct():
    words = []
    for c in range(4000):
        words.extend(PX.philox4x32_10((c, 7, 3, 1), (11, 13)))
    u = np.array([PX.u32(w) for w in words])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # distinct keys give unrelated streams
    w2 = [PX.philox4x32_10((c, 7, 3, 1), (12, 13))[0] for c in range(2000)]
    assert np.corrcoef(np.array(words[0:8000:4], dtype=float), np.array(w2, dtype=float))[0, 1] < 0.1
    # exact conversions
    assert PX.u53(0, 0) == 0.0 and PX.u53(0xFFFFFFFF, 0xFFFFFFFF) < 1.0
    assert PX.ranged(0xFFFFFFFF, 7) == 6 and PX.ranged(0, 7) == 0


def test_philox_known_answers():
    # the generator's published known-answer vectors (tests/golden/philox4x32_10_kat.json):
    # a wrong multiplier, Weyl constant, round count or word permutation changes every word
    import json
    import os
    kat = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        assert list(PX.philox4x32_10(ctr, key)) == [int(x, 16) for x in v["out"]]


def test_fdot_prior_is_the_one_induced_by_a_uniform_chirp_mass():
    # Mc ~ U[mc_min, mc_max] at fixed f0 gives p(fdot | f0) = |dMc/dfdot| / (mc_max - mc_min):
    # the sampler's prior ratio must equal the ratio of that Jacobian, here taken by central
    # finite differences of the chirp mass (whose formula the input-recipe test holds against
    # the recipe's own GR chirp); the support is the Mc interval, read back through Mc
    g = np.random.default_rng(40)
    cfg, _, _, _ = small_ensemble(seed=1, n_temps=1, n_walkers=1, n_bands=1, n_max=1, n_per_band=1, betas=(1.0,))

    def jac(f0, fd):
        h = 1e-6 * fd
        return (OM.chirp_mass(f0, fd + h) - OM.chirp_mass(f0, fd - h)) / (2 * h)

    lo, hi = cfg.allowance(0)
    for _ in range(200):
        f0a, f0b = g.uniform(lo, hi, 2)
        fa = OM.fdot_from_mc(f0a, g.uniform(0.3, 0.8))
        fb = OM.fdot_from_mc(f0b, g.uniform(0.3, 0.8))
        th = [1e-22, f0a, fa, 0.1, 0.2, 0.3, 0.4, 0.5]
        new = [1e-22, f0b, fb, 0.1, 0.2, 0.3, 0.4, 0.5]
        want = math.log(jac(f0b, fb)) - math.log(jac(f0a, fa))
        assert abs(OM.dlog_prior(new, th) - want) < 1e-6
        assert abs(OM.log_prior_shape(new) - OM.log_prior_shape(th) - OM.dlog_prior(new, th)) < 1e-9
    for _ in range(400):
        f0 = g.uniform(lo, hi)
        mc = g.uniform(0.1, 1.0)
        if min(abs(mc - 0.3), abs(mc - 0.8)) < 1e-9:
            continue
        th = [1e-22, f0, OM.fdot_from_mc(f0, mc), 0.1, 0.2, 0.3, 0.4, 0.5]
        assert OM.in_support(cfg, th, 0) == (0.3 < mc < 0.8), mc
    th = [1e-22, 0.5 * (lo + hi), OM.fdot_from_mc(0.5 * (lo + hi), 0.5), 0.1, 0.2, 0.3, 0.4, 0.5]
    assert OM.in_support(cfg, th, 0)
    for k, v in ((0, 2e-23 * 0.4), (0, 10 ** -21.4), (5, 1.0001), (6, -1.0001), (1, hi), (1, lo - 1e-12)):
        bad = list(th)
        bad[k] = v
        assert not OM.in_support(cfg, bad, 0), (k, v)


def test_prior_only_sweeps_reproduce_occupancy_and_f0_prior():
    pi = 0.3
    cfg, state, _, _ = small_ensemble(seed=9, n_temps=1, n_walkers=1, n_bands=2, n_max=6, n_per_band=1,
                                      betas=(0.0,), log_occ_odds=math.log(pi / (1 - pi)))
    st = copy_state(state)
    occ, frel = [], []
    for k in range(40):
        OM.sweep(cfg, st, k, do_swap=False)
        if k >= 4:
            occ.append(st["exists"].mean())
            for b in range(cfg.n_bands):
                lo, hi = cfg.allowance(b)
                f = st["params"][0, 0, b, :, 1][st["exists"][0, 0, b]]
                frel.extend(((f - lo) / (hi - lo)).tolist())
    n = len(occ) * cfg.n_bands * cfg.n_max
    assert abs(np.mean(occ) - pi) < 4 * math.sqrt(pi * (1 - pi) / n)
    assert stats.kstest(np.asarray(frel), "uniform").pvalue > 1e-3


def _table(cfg, g, peaked=True):
    from test_oracle_mdn import raw_from
    from oracle import mdn as MD
    t = np.empty((cfg.n_walkers, cfg.n_bands, MD.N_OUT))
    for w in range(cfg.n_walkers):
        for b in range(cfg.n_bands):
            pi = g.dirichlet(np.ones(MD.N_COMP))
            mu = g.uniform(0.25, 0.45, (MD.N_COMP, MD.N_DIM))
            s = g.uniform(0.03, 0.08, (MD.N_COMP, MD.N_DIM)) if peaked else np.full((MD.N_COMP, MD.N_DIM), 0.3)
            t[w, b] = raw_from(pi, mu, s)
    return t


def test_learned_proposal_with_eps_one_is_the_prior_sweep():
    # eps = 1 draws every birth from the prior branch (the same words as the prior draw)
    # and q = 1: the trace must equal the plain sweep's, decision by decision.
    cfg, state, _, _ = small_ensemble(seed=4, n_temps=2, n_walkers=1, n_bands=2, n_max=3, n_per_band=1,
                                      betas=(1.0, 0.5))
    t_plain = OM.sweep(cfg, copy_state(state), 0)
    cfg.mdn_raw, cfg.mdn_eps = _table(cfg, np.random.default_rng(5)), 1.0
    t_mdn = OM.sweep(cfg, copy_state(state), 0)
    assert len(t_plain) == len(t_mdn)
    for a, b in zip(t_plain, t_mdn):
        assert a["accepted"] == b["accepted"] and a["params"] == b["params"]
        assert a["log_alpha"] == b["log_alpha"] or (math.isinf(a["log_alpha"]) and math.isinf(b["log_alpha"]))


def test_prior_only_sweeps_with_learned_proposal_keep_the_prior():
    # With beta = 0 the target is the prior. A peaked proposal (components near u = 0.35,
    # widths 0.03-0.08) used for births, deaths and half the in-model moves must leave
    # the occupancy and the unit-box marginals unchanged; a wrong sign or a missing q
    # factor piles the sources up where q is large.
    pi = 0.4
    cfg, state, _, _ = small_ensemble(seed=10, n_temps=1, n_walkers=1, n_bands=2, n_max=6, n_per_band=1,
                                      betas=(0.0,), log_occ_odds=math.log(pi / (1 - pi)))
    from oracle import mdn as MD
    cfg.mdn_raw, cfg.mdn_eps, cfg.mdn_inmodel = _table(cfg, np.random.default_rng(6)), 0.2, 0.5
    st = copy_state(state)
    occ, u = [], []
    for k in range(60):
        OM.sweep(cfg, st, k, do_swap=False)
        if k >= 4:
            occ.append(st["exists"].mean())
            for b in range(cfg.n_bands):
                for s in range(cfg.n_max):
                    if st["exists"][0, 0, b, s]:
                        u.append(MD.to_unit(cfg, b, st["params"][0, 0, b, s]))
    u = np.asarray(u)
    n = len(occ) * cfg.n_bands * cfg.n_max
    assert abs(np.mean(occ) - pi) < 4 * math.sqrt(pi * (1 - pi) / n) * 2   # x2: correlated sweeps
    for d in (0, 1, 2, 7):
        assert stats.kstest(u[:, d], "uniform").pvalue > 1e-3, d


def test_friends_window_holds_the_nearest_members():
    g = np.random.default_rng(30)
    for _ in range(200):
        G = int(g.integers(1, 60))
        fs = np.sort(g.uniform(0, 1, G))
        nf = int(g.integers(1, G + 1))
        f = float(g.uniform(-0.2, 1.2))
        s = OM.friends_start(fs, f, nf)
        assert 0 <= s and s + nf <= G
        win = set(range(s, s + nf))
        far_in = max(abs(fs[i] - f) for i in win)
        near_out = min([abs(fs[i] - f) for i in range(G) if i not in win], default=np.inf)
        assert far_in <= near_out


def test_group_stretch_is_reversible_with_the_same_friend_and_inverse_z():
    # Y from (X, j, z); then from Y with the same j and 1/z the map returns X (periodic
    # coordinates included), whenever the move was accepted as reversible.
    cfg, state, _, _ = small_ensemble(seed=31, n_temps=1, n_walkers=4, n_bands=2, n_max=4, n_per_band=2,
                                      betas=(1.0,))
    grp = OM.build_group(cfg, state)
    g = np.random.default_rng(32)
    fs, gp = grp[0]
    n_rev = 0
    for _ in range(300):
        th = list(gp[int(g.integers(len(fs)))] + np.array([0, 0.3 * OM.PX.u32(1) * 0, 0, 0.1, 0.1, 0, 0, 0.1]))
        th[3] %= 2 * math.pi
        th[4] %= math.pi
        th[7] %= 2 * math.pi
        wj, wz = int(g.integers(2 ** 32)), int(g.integers(2 ** 32))
        new, lnz = OM.group_stretch(cfg, grp[0], th, wj, wz)
        if lnz is None:
            continue
        n_rev += 1
        nf = min(cfg.n_friends, len(fs))
        j = OM.friends_start(fs, th[1], nf) + OM.PX.ranged(wj, nf)
        z = math.exp(lnz)
        y = [math.log(new[0])] + list(new[1:])
        xj = [math.log(gp[j][0])] + list(gp[j][1:])
        back = []
        for c in range(8):
            per = OM.STRETCH_PERIODS[c]
            if per is None:
                back.append(xj[c] + (y[c] - xj[c]) / z)
            else:
                back.append((xj[c] + OM._wrap_sym(y[c] - xj[c], per) / z) % per)
        back[0] = math.exp(back[0])
        np.testing.assert_allclose(back, th, rtol=1e-9, atol=1e-12)
    assert n_rev > 100


def test_group_stretch_keeps_a_known_target_stationary():
    # The move on its own: chains started from exact draws of a known target (independent
    # normals in the stretch coordinates ln A, f0, fdot, cos i, sin b; uniform phases) take
    # 8 MH steps each with group-stretch proposals (a fixed group of 40 target draws, 8
    # friends); the final states must still follow the target. A kernel that does not
    # leave the target invariant shifts them: dropping or doubling the z^(d-1) factor, or
    # the reverse-friend condition, planted in the oracle on the CPU, fails this.
    class C:
        n_friends, stretch_a = 8, 2.0
    g = np.random.default_rng(34)
    mu = np.array([math.log(2e-22), 2.5e-3, 1e-17, 0.0, 0.0, 0.1, -0.2, 0.0])
    sd = np.array([0.3, 3e-8, 2e-19, 0.0, 0.0, 0.15, 0.1, 0.0])
    per = OM.STRETCH_PERIODS

    def draw(n):
        x = g.normal(mu, np.where(sd > 0, sd, 1.0), (n, 8))
        for c in range(8):
            if per[c] is not None:
                x[:, c] = g.uniform(0, per[c], n)
        return x

    def logp(u):
        return -0.5 * float(np.sum(((u - mu) / np.where(sd > 0, sd, 1.0)) ** 2 * (sd > 0)))

    gu = draw(40)
    gu = gu[np.argsort(gu[:, 1])]
    gp = gu.copy()
    gp[:, 0] = np.exp(gu[:, 0])
    group = (gp[:, 1].copy(), gp)
    starts = draw(3000)
    final = np.empty_like(starts)
    moved = 0
    for i, x in enumerate(starts):
        th = list(x)
        th[0] = math.exp(x[0])
        for _ in range(8):
            new, lnz = OM.group_stretch(C, group, th, int(g.integers(2 ** 32)), int(g.integers(2 ** 32)))
            if lnz is None:
                continue
            un = np.array([math.log(new[0])] + list(new[1:]))
            uo = np.array([math.log(th[0])] + list(th[1:]))
            if math.log(g.uniform()) < logp(un) - logp(uo) + 7.0 * lnz:
                th = new
                moved += 1
        final[i] = [math.log(th[0])] + list(th[1:])
    assert moved > 3000 * 8 * 0.15
    for c in (0, 1, 2, 5, 6):
        assert stats.kstest((final[:, c] - mu[c]) / sd[c], "norm").pvalue > 1e-3, c
    for c in (3, 4, 7):
        assert stats.kstest(final[:, c] / per[c], "uniform").pvalue > 1e-3, c


def test_nearest_friend_selection_needs_the_reverse_condition():
    # The friend rule on its own, in one dimension (N(0, 1) target, group of 40 draws, 8
    # nearest friends, 20 steps from 20000 exact draws): with the reverse condition (the
    # auxiliary point must also be among the proposed point's friends) the spread stays 1;
    # without it the spread shrinks (to ~0.97, six standard errors). This pins the
    # acceptance rule that group_stretch applies.
    g = np.random.default_rng(1)
    grp = np.sort(g.normal(0, 1, 40))

    def run(cond):
        xs = g.normal(0, 1, 20000)
        for i in range(len(xs)):
            x = xs[i]
            for _ in range(20):
                j = OM.friends_start(grp, x, 8) + int(g.integers(8))
                z = (g.uniform() + 1.0) ** 2 / 2.0
                y = grp[j] + z * (x - grp[j])
                ok = True
                if cond:
                    s1 = OM.friends_start(grp, y, 8)
                    ok = s1 <= j < s1 + 8
                if ok and math.log(g.uniform()) < 0.5 * (x * x - y * y):
                    x = y
            xs[i] = x
        return xs

    se = 1.0 / math.sqrt(2 * 20000)
    assert abs(run(True).std() - 1.0) < 3 * se
    assert run(False).std() < 1.0 - 3 * se


def test_prior_only_sweeps_with_group_stretch_keep_the_prior():
    # beta = 0: the target is the prior. Group stretch moves (70 % of the in-model moves,
    # 6 friends, a fixed group) must keep the unit-box marginals uniform; dropping the
    # z^(d-1) factor (planted in the oracle, on the CPU) fails this.
    from oracle import mdn as MD
    pi = 0.5
    cfg, state, _, _ = small_ensemble(seed=33, n_temps=1, n_walkers=2, n_bands=2, n_max=4, n_per_band=2,
                                      betas=(0.0,), log_occ_odds=math.log(pi / (1 - pi)))
    cfg.group, cfg.group_frac, cfg.n_friends = OM.build_group(cfg, state), 0.7, 6
    cfg.props_per_source = 3.0
    st = copy_state(state)
    u = []
    for k in range(50):
        OM.sweep(cfg, st, k, do_swap=False)
        if k >= 5:
            for w in range(cfg.n_walkers):
                for b in range(cfg.n_bands):
                    for s in range(cfg.n_max):
                        if st["exists"][0, w, b, s]:
                            u.append(MD.to_unit(cfg, b, st["params"][0, w, b, s]))
    u = np.asarray(u)
    for d in (0, 2, 3, 5):
        assert stats.kstest(u[::3, d], "uniform").pvalue > 1e-3, d


def test_ladder_adaptation_balances_the_swap_rates():
    b = np.array([1.0, 1 / 1.2, 1 / 1.44, 1 / 1.728, 0.0])
    # equal acceptances: the ladder does not move
    np.testing.assert_allclose(OM.adapt_ladder(b, [0, 0.4, 0.4, 0.4, 0.4], 0), b, rtol=1e-14)
    # a rung pair that swaps more often than the next one widens its gap
    out = OM.adapt_ladder(b, [0, 0.9, 0.2, 0.4, 0.4], 0)
    assert 1 / out[1] - 1 > 1 / b[1] - 1
    assert out[0] == 1.0 and out[-1] == 0.0 and np.all(np.diff(out) < 0)
    # one step by hand: S_1 = ln(0.2) + (t0/(nu t0)) (0.9 - 0.2)
    assert abs(1 / out[1] - (1 + math.exp(math.log(0.2) + 0.01 * 0.7))) < 1e-13
    # the step size decays as t0 / (t + t0)
    late = OM.adapt_ladder(b, [0, 0.9, 0.2, 0.4, 0.4], 99000)
    assert abs(1 / late[1] - 1.2) < 0.02 * abs(1 / out[1] - 1.2)
    # iterated with rates that fall with the gap, the rates equalise
    g = np.random.default_rng(0)
    lad = b.copy()
    for it in range(3000):
        temps = 1 / lad[:-1]
        rates = [0.0] + [math.exp(-2.0 * (temps[i] - temps[i - 1])) for i in range(1, len(temps))] + [0.3]
        lad = OM.adapt_ladder(lad, rates, it, nu=10.0, t0=100.0)
    temps = 1 / lad[:-1]
    r = [math.exp(-2.0 * (temps[i] - temps[i - 1])) for i in range(1, len(temps))] + [0.3]
    assert max(r) - min(r) < 0.05, r


def _xfer_cfg(n_bands, n_max, n_temps=2, n_walkers=1):
    tobs, band_k0 = 31457280.0, 65536
    n_bins = (n_bands + 4) * 256
    return OM.SweepConfig(tobs=tobs, k0=band_k0 - 512, n_bins=n_bins, band_k0=band_k0, nb=256, n_bands=n_bands,
                          n_temps=n_temps, n_walkers=n_walkers, n_max=n_max, betas=np.ones((n_bands, n_temps)),
                          psd=np.ones((n_walkers, n_bins)), sigma=np.ones(8), f_min=1e-4, f_max=1e-2)


def _at(cfg, x):
    """Parameters of a source x bins above band_k0 (only f0 matters to the transfer)."""
    th = np.zeros(8)
    th[0] = 1e-22
    th[1] = (cfg.band_k0 + x) / cfg.tobs
    return th


def test_ownership_transfer_worked_example():
    # Sec. V.D: a cold source that ended in a neighbour's own bins moves to that band.
    # Bands of 256 bins: band 0 owns x in [0, 256), band 1 [256, 512), band 2 [512, 768).
    cfg = _xfer_cfg(3, 3)
    st = {"params": np.zeros((2, 1, 3, 3, 8)), "exists": np.zeros((2, 1, 3, 3), bool)}
    layout = {(0, 0): 100, (0, 1): 300, (0, 2): -50,     # band 0: own, band 1's, below band 0 (stays)
              (1, 0): 400, (1, 1): 450,                  # band 1: two own, slot 2 free
              (2, 0): 600, (2, 1): 500, (2, 2): 800}     # band 2: own, band 1's (blocked), beyond band 2
    for (b, s), x in layout.items():
        for t in range(2):
            st["params"][t, 0, b, s] = _at(cfg, x)
            st["exists"][t, 0, b, s] = True
    hot = (st["params"][1].copy(), st["exists"][1].copy())
    moved, blocked = OM.transfer_ownership(cfg, st)
    assert (moved, blocked) == (1, 1)
    E = st["exists"][0, 0]
    assert E.tolist() == [[True, False, True], [True, True, True], [True, True, True]]
    assert np.array_equal(st["params"][0, 0, 1, 2], _at(cfg, 300))
    assert np.array_equal(st["params"][0, 0, 2, 1], _at(cfg, 500))
    assert np.array_equal(st["params"][1], hot[0]) and np.array_equal(st["exists"][1], hot[1])
    # band 1 takes band 0's candidate before band 2's: with room for both, both move
    st["exists"][0, 0, 1, :2] = False
    st["exists"][0, 0, 0, 1] = True
    st["params"][0, 0, 0, 1] = _at(cfg, 260)
    assert OM.transfer_ownership(cfg, st) == (2, 0)
    assert np.array_equal(st["params"][0, 0, 1, 0], _at(cfg, 260))
    assert np.array_equal(st["params"][0, 0, 1, 1], _at(cfg, 500))
    assert st["exists"][0, 0].tolist() == [[True, False, True], [True, True, True], [True, False, True]]


def test_ownership_transfer_keeps_the_model_and_fills_owners():
    # Random cold states (sources anywhere in their band's allowance): the transfer keeps the
    # multiset of sources, never overfills a band, moves a source only into its owner; repeated
    # until nothing moves, every source sits in its owner band unless that band is full or
    # outside the range.
    g = np.random.default_rng(5)
    for trial in range(20):
        n_bands, n_max, W = 6, 4, 3
        cfg = _xfer_cfg(n_bands, n_max, n_temps=1, n_walkers=W)
        st = {"params": np.zeros((1, W, n_bands, n_max, 8)), "exists": g.uniform(size=(1, W, n_bands, n_max)) < 0.6}
        for w in range(W):
            for b in range(n_bands):
                for s in range(n_max):
                    st["params"][0, w, b, s] = _at(cfg, 256 * b + g.uniform(-128, 384))
        before = sorted(tuple(st["params"][0, w, b, s]) + (w,) for w, b, s in zip(*np.nonzero(st["exists"][0])))
        total = 0
        for _ in range(10):
            prev = st["exists"][0].copy(), st["params"][0].copy()
            moved, _ = OM.transfer_ownership(cfg, st)
            total += moved
            for w, b, s in zip(*np.nonzero(st["exists"][0] & ~prev[0])):    # arrivals sit in their owner
                assert OM.owner_band(cfg, st["params"][0, w, b, s, 1]) == b
            if moved == 0:
                break
        after = sorted(tuple(st["params"][0, w, b, s]) + (w,) for w, b, s in zip(*np.nonzero(st["exists"][0])))
        assert before == after
        assert total > 0 or trial > 0
        for w, b, s in zip(*np.nonzero(st["exists"][0])):
            o = OM.owner_band(cfg, st["params"][0, w, b, s, 1])
            assert abs(o - b) <= 1
            assert o == b or not 0 <= o < n_bands or st["exists"][0, w, o].all()
