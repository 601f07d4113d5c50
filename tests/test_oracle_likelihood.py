"""Pins of the oracle's inner products and Delta log-likelihoods (Eq. like, inner,
addsource, swapsource) and of the fixed-point residual."""
import numpy as np

from oracle import constants as C
from oracle import likelihood as LK
from oracle import psd as P
from oracle import residual as RS
from oracle import waveform as W
from paper_2405_04690_gb300 import synth

N = 256


def _setup(seed, n_src=3, noise=True):
    g = synth.rng(seed)
    p = synth.draw_sources(g, n_src, 2.0e-3, 2.004e-3)
    k0 = int(np.floor(2.0e-3 * C.TOBS)) - 600
    n = 1400
    f = (k0 + np.arange(n)) * C.DF
    s = P.psd_ae(f, C.SQRT_S_OMS, C.SQRT_S_ACC)
    d = np.zeros((2, n), complex)
    if noise:
        d += synth.unit_complex_normal(g, (2, n)) * np.sqrt(s / (4 * C.DF))
    bands = [W.fastslow_band(p[:, i], N) for i in range(n_src)]
    return g, p, k0, n, s, d, bands


def test_propose_injected_source_gives_half_snr2():
    # Invariant (d): data = h (no noise), model empty; adding h gives +1/2 <h|h>.
    _, p, k0, n, s, _, bands = _setup(21, 1, noise=False)
    h = LK.place(bands[0], k0, n)
    dll = LK.delta_loglike_swap(h, s, C.DF, k0, bands[0], None)
    snr2 = LK.inner(h, h, s, C.DF)
    assert snr2 > 1.0
    assert abs(dll - 0.5 * snr2) <= 1e-12 * snr2


def test_swap_with_zero_template_is_addsource():
    _, p, k0, n, s, d, bands = _setup(22)
    a = LK.place(bands[0], k0, n)
    add = -0.5 * (LK.inner(a, a, s, C.DF) - 2 * LK.inner(d, a, s, C.DF))   # Eq. addsource
    assert abs(LK.delta_loglike_swap(d, s, C.DF, k0, bands[0], None) - add) < 1e-10 * max(1, abs(add))


def test_difference_form_equals_expanded_and_bruteforce():
    _, p, k0, n, s, d, bands = _setup(23)
    resid = d - LK.place(bands[1], k0, n) - LK.place(bands[2], k0, n)
    for new, old in ((bands[0], bands[1]), (bands[0], None), (None, bands[2]), (bands[2], bands[1])):
        e = LK.delta_loglike_swap(resid, s, C.DF, k0, new, old)
        dif = LK.delta_loglike_difference(resid, s, C.DF, k0, new, old)
        bf = LK.delta_loglike_bruteforce(resid, s, C.DF, k0, new, old)
        scale = max(1.0, abs(e))
        assert abs(e - dif) < 1e-10 * scale
        assert abs(e - bf) < 1e-8 * scale


def test_zero_amplitude_proposal_has_zero_delta():
    # Invariant (a) at the likelihood level: a template of amplitude 0 changes nothing.
    _, p, k0, n, s, d, _ = _setup(24, 1)
    q = p[:, 0].copy()
    q[0] = 0.0
    z = W.fastslow_band(q, N)
    assert LK.delta_loglike_swap(d, s, C.DF, k0, z, None) == 0.0


def test_loglike_white_psd_closed_form():
    # Eq. like with constant S: -1/2 * 4 df sum |R|^2 / S - 2 n ln S.
    g = synth.rng(25)
    n = 1000
    r = synth.unit_complex_normal(g, (2, n)) * 1e-18
    s0 = 3e-40
    expect = -0.5 * 4 * C.DF * np.sum(np.abs(r) ** 2) / s0 - 2 * n * np.log(s0)
    got = LK.loglike(r, np.full(n, s0), C.DF)
    assert abs(got - expect) < 1e-12 * abs(expect)


def test_fixed_point_inject_then_subtract_is_bitwise():
    # Invariant (c).
    g, p, k0, n, s, d, bands = _setup(26)
    frac = 98
    r0 = RS.to_fixed(d, frac)
    r = r0
    for b in bands:
        r = RS.add_sub(r, k0, b, +1, frac)
    for b in reversed(bands):
        r = RS.add_sub(r, k0, b, -1, frac)
    assert np.array_equal(r, r0)
    # order independence of integer add/sub
    r1 = RS.add_sub(RS.add_sub(r0, k0, bands[0], +1, frac), k0, bands[1], +1, frac)
    r2 = RS.add_sub(RS.add_sub(r0, k0, bands[1], +1, frac), k0, bands[0], +1, frac)
    assert np.array_equal(r1, r2)
    # three roundings (data and two templates), each at most half a unit of 2^-frac
    # per component
    back = RS.from_fixed(r1, frac)
    exact = d - LK.place(bands[0], k0, n) - LK.place(bands[1], k0, n)
    assert np.max(np.abs(back.real - exact.real)) <= 1.5 * 2.0 ** -frac * (1 + 1e-9)
    assert np.max(np.abs(back.imag - exact.imag)) <= 1.5 * 2.0 ** -frac * (1 + 1e-9)
