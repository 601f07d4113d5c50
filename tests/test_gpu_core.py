"""GPU parity of the C-ABI calls against the FP64 oracle (seeded inputs).

Tolerances: waveform relative L2 < 1e-5 (mixed) and < 1e-11 (FP64) per source;
|Delta lnL error| < 1e-2 (mixed) and < 1e-7 (FP64); integer results bit-exact.
"""
import numpy as np
import pytest

from oracle import constants as OC
from oracle import likelihood as OL
from oracle import psd as OP
from oracle import residual as OR
from oracle import waveform as OW
from paper_2405_04690_gb300 import synth

from _common import FRAC_BITS, noise_fixed, psd_window, rel_l2, torch_cuda, window

pytestmark = pytest.mark.gpu

WF_TOL = {"mixed": 1e-5, "fp64": 1e-11}
DLL_TOL = {"mixed": 1e-2, "fp64": 1e-7}


def _ctx(L, k0, n):
    return L.Context(OC.TOBS, OC.DT, k0, n)


def _band_for(f0):
    return 128 if f0 < 1e-3 else 256 if f0 < 2e-3 else 512 if f0 < 4e-3 else 1024


def _run_waveforms(torch, L, ctx, p, nb, prec):
    dev = torch.device("cuda")
    n = p.shape[1]
    off = np.concatenate([[0], np.cumsum(nb)[:-1]]).astype(np.int64)
    cdt = torch.complex64 if prec == "mixed" else torch.complex128
    ha = torch.zeros(int(nb.sum()), dtype=cdt, device=dev)
    he = torch.zeros_like(ha)
    ks = torch.zeros(n, dtype=torch.int64, device=dev)
    L.gb_waveform_batch(ctx, torch.from_numpy(p).to(dev), torch.from_numpy(nb.astype(np.int32)).to(dev),
                        int(nb.max()), ks, ha, he, torch.from_numpy(off).to(dev), L.PRECISION[prec])
    L.gbk_sync_status(ctx)
    return ks.cpu().numpy(), ha.cpu().numpy(), he.cpu().numpy(), off


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_waveform_matches_oracle_n256(prec):
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(0)
    p = synth.draw_sources(g, 64)
    k0, n = window()
    ctx = _ctx(L, k0, n)
    nb = np.full(64, 256)
    ks, ha, he, off = _run_waveforms(torch, L, ctx, p, nb, prec)
    worst = 0.0
    for i in range(64):
        k, a, e = OW.fastslow_band(p[:, i], 256)
        assert ks[i] == k
        got = np.concatenate([ha[off[i]:off[i] + 256], he[off[i]:off[i] + 256]])
        worst = max(worst, rel_l2(got, np.concatenate([a, e])))
    assert worst < WF_TOL[prec], worst


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_waveform_ragged_band_lengths(prec):
    # f0 log-uniform over 0.3-20 mHz with N doubling per octave: one batch, all four N.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(2)
    p = synth.draw_sources(g, 37, 3e-4, 2e-2, log_f=True)
    nb = np.array([_band_for(f) for f in p[1]])
    k0, n = window(2.5e-4, 2.1e-2, 700)
    ctx = _ctx(L, k0, n)
    ks, ha, he, off = _run_waveforms(torch, L, ctx, p, nb, prec)
    for i in range(p.shape[1]):
        k, a, e = OW.fastslow_band(p[:, i], int(nb[i]))
        assert ks[i] == k
        got = np.concatenate([ha[off[i]:off[i] + nb[i]], he[off[i]:off[i] + nb[i]]])
        assert rel_l2(got, np.concatenate([a, e])) < WF_TOL[prec]


def test_waveform_on_both_sides_of_the_short_series_limit():
    # The float generator evaluates shorter series for sources whose largest series argument
    # 2 pi f_max L/c is at most 0.25 rad (f below 4.77 mHz over the observation); sources just
    # below and just above that frequency match the oracle alike, and neither side is worse.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(7)
    p = synth.draw_sources(g, 48, 4.55e-3, 5.0e-3)
    f_max = np.maximum(np.abs(p[1]), np.abs(p[1] + p[2] * OC.TOBS))
    short = 2.0 * np.pi * f_max * OC.L_ARM / OC.C_LIGHT <= 0.25
    assert 8 <= short.sum() <= 40
    nb = np.full(48, 512)
    k0, n = window(4.5e-3, 5.05e-3, 700)
    ctx = _ctx(L, k0, n)
    ks, ha, he, off = _run_waveforms(torch, L, ctx, p, nb, "mixed")
    err = np.empty(48)
    for i in range(48):
        k, a, e = OW.fastslow_band(p[:, i], 512)
        assert ks[i] == k
        err[i] = rel_l2(np.concatenate([ha[off[i]:off[i] + 512], he[off[i]:off[i] + 512]]), np.concatenate([a, e]))
    assert err.max() < WF_TOL["mixed"], err.max()
    assert np.median(err[short]) < 2.0 * np.median(err[~short]), (np.median(err[short]), np.median(err[~short]))


def test_waveform_invariants_on_gpu():
    # (a) A = 0 gives exact zeros; (b) phi0 + pi negates the band.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(3)
    p = synth.draw_sources(g, 4)
    z = p.copy()
    z[0] = 0.0
    s = p.copy()
    s[3] += np.pi
    k0, n = window()
    ctx = _ctx(L, k0, n)
    nb = np.full(4, 256)
    for prec in ("mixed", "fp64"):
        _, za, ze, _ = _run_waveforms(torch, L, ctx, z, nb, prec)
        assert np.all(za == 0) and np.all(ze == 0)
        _, ha, he, _ = _run_waveforms(torch, L, ctx, p, nb, prec)
        _, sa, se, _ = _run_waveforms(torch, L, ctx, s, nb, prec)
        tol = 1e-5 if prec == "mixed" else 1e-12
        assert rel_l2(np.concatenate([sa, se]), -np.concatenate([ha, he])) < tol


def _config0(seed=0, n_src=64, per_src=16):
    """64 injected sources in noise; 16 Gaussian in-model proposals per source."""
    g = synth.rng(seed)
    p = synth.draw_sources(g, n_src)
    k0, n = window()
    s = psd_window(k0, n)
    rfix = noise_fixed(g, k0, n, s)
    old = np.repeat(p, per_src, axis=1)
    new = synth.perturb(g, old, synth.proposal_widths(old))
    return g, p, k0, n, s, rfix, old, new


def _oracle_dlogl(rfix, s, k0, new, old, nb=256):
    r = OR.from_fixed(rfix, FRAC_BITS)
    out = np.empty(new.shape[1])
    for i in range(new.shape[1]):
        bn = OW.fastslow_band(new[:, i], nb) if new[0, i] != 0 else None
        bo = OW.fastslow_band(old[:, i], nb) if old[0, i] != 0 else None
        out[i] = OL.delta_loglike_swap(r, s, OC.DF, k0, bn, bo)
    return out


def _gpu_dlogl(torch, L, ctx, rfix_w, psdp, new, old, walker, prec, nb=256):
    dev = torch.device("cuda")
    resid = torch.from_numpy(np.ascontiguousarray(rfix_w)).to(dev)
    pp = torch.from_numpy(np.ascontiguousarray(psdp)).to(dev)
    m = new.shape[1]
    out = torch.empty(m, dtype=torch.float64, device=dev)
    L.gb_delta_loglike_batch(ctx, torch.from_numpy(new).to(dev), torch.from_numpy(old).to(dev),
                             torch.full((m,), nb, dtype=torch.int32, device=dev), nb,
                             torch.from_numpy(walker.astype(np.int32)).to(dev),
                             L.residual_struct(resid, FRAC_BITS), L.psd_struct(pp), out, L.PRECISION[prec])
    L.gbk_sync_status(ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_dlogl_config0_in_model(prec):
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    _, p, k0, n, s, rfix, old, new = _config0(per_src=4)
    want = _oracle_dlogl(rfix, s, k0, new, old)
    ctx = _ctx(L, k0, n)
    got = _gpu_dlogl(torch, L, ctx, rfix[None], np.array([[OC.SQRT_S_OMS, OC.SQRT_S_ACC]]), new, old,
                     np.zeros(new.shape[1]), prec)
    err = np.max(np.abs(got - want))
    assert err < DLL_TOL[prec], err


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_dlogl_birth_death_and_degenerate(prec):
    # birth (old A = 0), death (new A = 0), both zero (exactly 0), identical (exactly 0)
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g, p, k0, n, s, rfix, old, new = _config0(seed=5, n_src=16, per_src=1)
    births_old = old.copy(); births_old[0] = 0.0
    deaths_new = new.copy(); deaths_new[0] = 0.0
    both_new = deaths_new.copy(); both_old = births_old.copy()
    cat_new = np.concatenate([new, deaths_new, both_new, old], axis=1)
    cat_old = np.concatenate([births_old, old, both_old, old], axis=1)
    want = _oracle_dlogl(rfix, s, k0, cat_new, cat_old)
    ctx = _ctx(L, k0, n)
    got = _gpu_dlogl(torch, L, ctx, rfix[None], np.array([[OC.SQRT_S_OMS, OC.SQRT_S_ACC]]), cat_new, cat_old,
                     np.zeros(cat_new.shape[1]), prec)
    assert np.max(np.abs(got - want)) < DLL_TOL[prec]
    assert np.all(got[32:48] == 0.0)      # both templates zero
    assert np.all(got[48:] == 0.0)        # a == r exactly: Delta = 0 bitwise


def test_dlogl_injected_source_noise_free_is_half_snr2():
    # Invariant (d) through the GPU: residual = h (no noise, empty model), birth of h.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(8)
    p = synth.draw_sources(g, 8)
    k0, n = window()
    s = psd_window(k0, n)
    ctx = _ctx(L, k0, n)
    for i in range(8):
        band = OW.fastslow_band(p[:, i], 256)
        h = OL.place(band, k0, n)
        rfix = OR.to_fixed(h, FRAC_BITS)
        snr2 = OL.inner(h, h, s, OC.DF)
        old = p[:, i:i + 1].copy(); old[0] = 0.0
        for prec in ("mixed", "fp64"):
            got = _gpu_dlogl(torch, L, ctx, rfix[None], np.array([[OC.SQRT_S_OMS, OC.SQRT_S_ACC]]), p[:, i:i + 1],
                             old, np.zeros(1), prec)[0]
            assert abs(got - 0.5 * snr2) < DLL_TOL[prec] + 1e-9 * snr2


def test_dlogl_many_walkers_own_psd():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(9)
    nw = 5
    k0, n = window()
    psdp = synth.draw_psd_params(g, nw)
    res, ss = [], []
    for w in range(nw):
        s = psd_window(k0, n, psdp[w, 0], psdp[w, 1])
        ss.append(s)
        res.append(noise_fixed(g, k0, n, s))
    p = synth.draw_sources(g, 20)
    new = synth.perturb(g, p, synth.proposal_widths(p))
    walker = g.integers(0, nw, 20)
    ctx = _ctx(L, k0, n)
    for prec in ("mixed", "fp64"):
        got = _gpu_dlogl(torch, L, ctx, np.stack(res), psdp, new, p, walker, prec)
        for i in range(20):
            w = walker[i]
            want = _oracle_dlogl(res[w], ss[w], k0, new[:, i:i + 1], p[:, i:i + 1])[0]
            assert abs(got[i] - want) < DLL_TOL[prec]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_residual_add_sub_bit_exact_and_matches_oracle(prec):
    # Invariant (c) on the GPU, overlapping templates in one walker (integer atomics),
    # and the injected values against the oracle's rounded waveform.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(10)
    k0, n = window(2.0e-3, 2.01e-3, 600)
    s = psd_window(k0, n)
    rfix = np.stack([noise_fixed(g, k0, n, s), noise_fixed(g, k0, n, s)])
    p = synth.draw_sources(g, 40, 2.0e-3, 2.01e-3)       # heavily overlapping bands
    walker = (np.arange(40) % 2).astype(np.int32)
    dev = torch.device("cuda")
    r = torch.from_numpy(rfix.copy()).to(dev)
    R = L.residual_struct(r, FRAC_BITS)
    ctx = _ctx(L, k0, n)
    pt = torch.from_numpy(p).to(dev)
    nb = torch.full((40,), 256, dtype=torch.int32, device=dev)
    wt = torch.from_numpy(walker).to(dev)
    L.residual_add_sub(ctx, R, pt, nb, 256, wt, +1, L.PRECISION[prec])
    L.gbk_sync_status(ctx)
    after = r.cpu().numpy()
    # injected signal vs oracle
    for w in range(2):
        delta = OR.from_fixed(rfix[w], FRAC_BITS) - OR.from_fixed(after[w], FRAC_BITS)
        want = sum(OL.place(OW.fastslow_band(p[:, i], 256), k0, n) for i in range(40) if walker[i] == w)
        assert rel_l2(delta, want) < WF_TOL[prec] + 2e-12
    # remove in a different order: bit-exact restore
    perm = g.permutation(40)
    L.residual_add_sub(ctx, R, torch.from_numpy(np.ascontiguousarray(p[:, perm])).to(dev), nb, 256,
                       torch.from_numpy(walker[perm].copy()).to(dev), -1, L.PRECISION[prec])
    L.gbk_sync_status(ctx)
    assert np.array_equal(r.cpu().numpy(), rfix)


def test_psd_eval_matches_oracle():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(11)
    k0, n = 3146, 1 << 16
    psdp = synth.draw_psd_params(g, 3)
    ctx = _ctx(L, k0, n)
    dev = torch.device("cuda")
    out = torch.empty((3, n), dtype=torch.float64, device=dev)
    L.psd_eval(ctx, torch.from_numpy(psdp).to(dev), out)
    L.gbk_sync_status(ctx)
    got = out.cpu().numpy()
    for w in range(3):
        want = psd_window(k0, n, psdp[w, 0], psdp[w, 1])
        np.testing.assert_allclose(got[w], want, rtol=1e-12)


def test_total_loglike_matches_oracle():
    # Eq. like per walker; n odd to exercise the scalar tail, several walker groups.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(12)
    k0, n = 3146, 50001
    nw = 11
    psdp = synth.draw_psd_params(g, nw)
    R = np.empty((nw, 2, n), complex)
    want = np.empty(nw)
    for w in range(nw):
        s = psd_window(k0, n, psdp[w, 0], psdp[w, 1])
        R[w] = synth.unit_complex_normal(g, (2, n)) * np.sqrt(s / (4 * OC.DF))
        R[w] = R[w].astype(np.complex64)          # the GPU input is float32
        want[w] = OL.loglike(R[w], s, OC.DF)
    dev = torch.device("cuda")
    rt = torch.from_numpy(R.astype(np.complex64)).view(torch.float32).reshape(nw, 2, n, 2).to(dev)
    out = torch.empty(nw, dtype=torch.float64, device=dev)
    ctx = _ctx(L, k0, n)
    L.total_loglike(ctx, rt.contiguous(), torch.from_numpy(psdp).to(dev), out)
    L.gbk_sync_status(ctx)
    got = out.cpu().numpy()
    # float32 per-bin terms: each of the ~3n terms of size O(1) carries <= 2^-22 relative
    # error, so |error| <= 3 n 2^-22 (~0.04 here); compensated sums add nothing.
    tol = 3 * n * 2.0 ** -22
    assert np.max(np.abs(got - want)) < tol, (np.max(np.abs(got - want)), tol)


def test_total_loglike_full_window_has_no_systematic_error():
    # The bench's window (2^20 bins from k0 = 3146) with residuals whose noise is off their
    # walker's PSD by up to 30 %: then an error of the PSD that is the same in every bin (for
    # example the float32 rounding of S_acc / S_oms) no longer cancels between -1/2 <R|R> and
    # -sum ln S. The per-bin rounding of the float32 terms is random and sums to ~1e-4 here.
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    g = synth.rng(14)
    k0, n, nw = 3146, 1 << 20, 4
    psdp = synth.draw_psd_params(g, nw)
    R = np.empty((nw, 2, n), np.complex64)
    want = np.empty(nw)
    for w, scale in enumerate((0.7, 0.9, 1.1, 1.3)):
        s = psd_window(k0, n, psdp[w, 0], psdp[w, 1])
        R[w] = (scale * synth.unit_complex_normal(g, (2, n)) * np.sqrt(s / (4 * OC.DF))).astype(np.complex64)
        want[w] = OL.loglike(R[w].astype(np.complex128), s, OC.DF)
    dev = torch.device("cuda")
    rt = torch.from_numpy(R).view(torch.float32).reshape(nw, 2, n, 2).contiguous().to(dev)
    out = torch.empty(nw, dtype=torch.float64, device=dev)
    ctx = _ctx(L, k0, n)
    L.total_loglike(ctx, rt, torch.from_numpy(psdp).to(dev), out)
    L.gbk_sync_status(ctx)
    err = np.abs(out.cpu().numpy() - want)
    assert np.max(err) < 5e-3, (err, want)


def test_errors_are_reported_not_faulted():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    k0, n = window(2e-3, 2.1e-3, 200)
    ctx = _ctx(L, k0, n)
    dev = torch.device("cuda")
    g = synth.rng(13)
    p = synth.draw_sources(g, 3, 3.5e-3, 3.6e-3)            # far outside the window
    r = torch.zeros((1, 2, n, 2), dtype=torch.int64, device=dev)
    pp = torch.tensor([[OC.SQRT_S_OMS, OC.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    pt = torch.from_numpy(p).to(dev)
    nb = torch.full((3,), 256, dtype=torch.int32, device=dev)
    w = torch.zeros(3, dtype=torch.int32, device=dev)
    L.gb_delta_loglike_batch(ctx, pt, pt, nb, 256, w, L.residual_struct(r, FRAC_BITS), L.psd_struct(pp), out,
                             L.GBK_MIXED)
    with pytest.raises(L.GbkError) as ei:
        L.gbk_sync_status(ctx)
    assert ei.value.status == 2
    assert np.all(np.isnan(out.cpu().numpy()))
    # unsupported band length in the batch -> reported, nothing written out of bounds
    nb_bad = torch.tensor([256, 300, 256], dtype=torch.int32, device=dev)
    L.residual_add_sub(ctx, L.residual_struct(r, FRAC_BITS), pt, nb_bad, 256, w, +1, L.GBK_MIXED)
    with pytest.raises(L.GbkError):
        L.gbk_sync_status(ctx)
    assert int(r.abs().sum()) == 0
    # host-side argument errors
    with pytest.raises(L.GbkError):
        L.residual_add_sub(ctx, L.residual_struct(r, FRAC_BITS), pt, nb, 200, w, +1, L.GBK_MIXED)
    with pytest.raises(L.GbkError):
        L.residual_add_sub(ctx, L.residual_struct(r, FRAC_BITS), pt, nb, 256, w, 2, L.GBK_MIXED)
    # empty batches are fine
    e0 = torch.zeros((8, 0), dtype=torch.float64, device=dev)
    L.gb_delta_loglike_batch(ctx, e0, e0, nb[:0], 256, w[:0], L.residual_struct(r, FRAC_BITS), L.psd_struct(pp),
                             out[:0], L.GBK_MIXED)
    L.gbk_sync_status(ctx)
