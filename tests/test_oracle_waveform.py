"""Pins of the oracle waveform: fast/slow (W2) against the brute-force response (W1),
invariants (a) and (b), linearity, Parseval, the long-wavelength limit, and the textbook
sky- and polarisation-averaged antenna pattern (3/20 for 60-degree arms)."""
import numpy as np
import pytest

from oracle import constants as C
from oracle import orbits as O
from oracle import waveform as W
from paper_2405_04690_gb300 import synth

NT_TINY = 2 ** 16
DT = 15.0
T_TINY = NT_TINY * DT


def _rel_l2(a1, e1, a2, e2):
    num = np.sum(np.abs(a1 - a2) ** 2) + np.sum(np.abs(e1 - e2) ** 2)
    den = np.sum(np.abs(a2) ** 2) + np.sum(np.abs(e2) ** 2)
    return np.sqrt(num / den)


@pytest.mark.slow
def test_fastslow_matches_bruteforce_tiny_tobs():
    # Invariant (e): W2 agrees with the folded direct DFT of the exact response to 1e-3.
    g = synth.rng(11)
    p = synth.draw_sources(g, 12)
    t = np.arange(NT_TINY) * DT
    worst = 0.0
    for i in range(p.shape[1]):
        za, ze = W.bruteforce_tdi(p[:, i], t)
        q, _ = W.carrier_bin(p[1, i], T_TINY)
        spec_a = np.fft.fft(za) * DT
        spec_e = np.fft.fft(ze) * DT
        for n in (64, 128, 256):
            k2, a2, e2 = W.fastslow_band(p[:, i], n, T_TINY)
            bins = (q - n // 2 + np.arange(n)) % n
            a1 = 0.5 * spec_a.reshape(-1, n).sum(axis=0)[bins]
            e1 = 0.5 * spec_e.reshape(-1, n).sum(axis=0)[bins]
            assert k2 == q - n // 2
            worst = max(worst, _rel_l2(a2, e2, a1, e1))
    assert worst < 1e-3
    # the approximation error is that of slow geometry over the TDI delays, ~1e-4
    assert worst < 2e-4


@pytest.mark.slow
def test_fastslow_matches_bruteforce_full_year():
    g = synth.rng(12)
    p = synth.draw_sources(g, 1)[:, 0]
    k1, a1, e1 = W.bruteforce_band(p, 256, C.N_T, C.DT, fold=True)
    k2, a2, e2 = W.fastslow_band(p, 256)
    assert k1 == k2
    assert _rel_l2(a2, e2, a1, e1) < 1e-3


def test_band_truncation_leakage_is_information_only():
    # Without folding, the band misses the sinc tails of a tone that is not
    # bin-centred; this is inherent to band truncation and only bounded here.
    g = synth.rng(13)
    p = synth.draw_sources(g, 2)
    for i in range(2):
        k1, a1, e1 = W.bruteforce_band(p[:, i], 128, NT_TINY, DT, fold=False)
        k2, a2, e2 = W.fastslow_band(p[:, i], 128, T_TINY)
        assert _rel_l2(a2, e2, a1, e1) < 0.2


def test_zero_amplitude_gives_zero_bitwise():
    # Invariant (a).
    g = synth.rng(14)
    p = synth.draw_sources(g, 3)
    p[0] = 0.0
    for i in range(3):
        _, a, e = W.fastslow_band(p[:, i], 256)
        assert np.all(a == 0) and np.all(e == 0)


def test_phase_shift_by_pi_negates():
    # Invariant (b): h(phi0 + pi) = -h, to 1e-12 relative in FP64.
    g = synth.rng(15)
    p = synth.draw_sources(g, 4)
    for i in range(4):
        _, a, e = W.fastslow_band(p[:, i], 256)
        q = p[:, i].copy()
        q[3] += np.pi
        _, a2, e2 = W.fastslow_band(q, 256)
        assert _rel_l2(a2, e2, -a, -e) < 1e-12


def test_linear_in_amplitude():
    g = synth.rng(16)
    p = synth.draw_sources(g, 1)[:, 0]
    _, a, e = W.fastslow_band(p, 256)
    q = p.copy()
    q[0] *= 3.0
    _, a3, e3 = W.fastslow_band(q, 256)
    assert _rel_l2(a3, e3, 3 * a, 3 * e) < 1e-14


def test_parseval_of_bruteforce_spectrum():
    # Eq. inner with a white PSD: 4 df sum_k |x~_k|^2 / S = 2 dt sum_n x_n^2 / S for the
    # real signal x = Re z; the positive-frequency spectrum is half the analytic one.
    g = synth.rng(17)
    p = synth.draw_sources(g, 1)[:, 0]
    t = np.arange(NT_TINY) * DT
    za, _ = W.bruteforce_tdi(p, t)
    spec = 0.5 * np.fft.fft(za) * DT
    lhs = 4.0 / T_TINY * np.sum(np.abs(spec) ** 2)
    rhs = 2.0 * DT * np.sum(za.real ** 2)
    assert abs(lhs / rhs - 1) < 1e-3


def test_long_wavelength_limit():
    # For u = 2 pi f L / c << 1 the slow part of X tends to the Michelson strain
    # difference 2 u^2 (n13.H.n13 - n12.H.n12) e^{-2 pi i f k.x1 / c}, and Y, Z by the
    # cyclic map; the relative correction is O(u).
    t = np.linspace(0, C.TOBS, 64, endpoint=False)
    x = O.spacecraft_positions(t)
    errs = []
    for f0 in (2e-5, 2e-6):
        p = np.array([1e-22, f0, 0.0, 0.3, 0.7, 0.4, 0.2, 1.1])
        X, Y, Z = W.slow_tdi(p, t)
        # independent construction of the tensor amplitude and the arm projections
        cb = np.sqrt(1 - 0.2 ** 2)
        kvec = -np.array([cb * np.cos(1.1), cb * np.sin(1.1), 0.2])
        uu = np.array([0.2 * np.cos(1.1), 0.2 * np.sin(1.1), -cb])
        vv = np.array([np.sin(1.1), -np.cos(1.1), 0.0])
        c2, s2 = np.cos(1.4), np.sin(1.4)
        def proj(n):
            un, vn = uu @ n, vv @ n
            plus, cross = un * un - vn * vn, 2 * un * vn
            return (1e-22 * (1 + 0.16) * (c2 * plus - s2 * cross)
                    + 2j * 1e-22 * 0.4 * (s2 * plus + c2 * cross))
        u = 2 * np.pi * f0 * C.L_ARM / C.C_LIGHT
        worst = 0.0
        for S, a, b, c in ((X, 0, 1, 2), (Y, 1, 2, 0), (Z, 2, 0, 1)):
            nab = O.arm_unit(x[a], x[b])
            nac = O.arm_unit(x[a], x[c])
            lw = 2 * u * u * (proj(nac) - proj(nab)) * np.exp(-2j * np.pi * f0 * (kvec @ x[a]) / C.C_LIGHT)
            worst = max(worst, np.max(np.abs(S - lw)) / np.max(np.abs(lw)))
        errs.append((u, worst))
    for u, w in errs:
        assert w < 4 * u
    # error shrinks in proportion to u
    assert errs[1][1] < 0.2 * errs[0][1]


def test_sky_and_polarisation_averaged_response():
    # Textbook antenna pattern of a two-arm interferometer with opening angle gamma (60 deg here):
    # averaged over an isotropic sky and the polarisation angle, <F+^2> = <Fx^2> = sin^2(gamma)/5
    # = 3/20 and <F+ Fx> = 0. In the long-wavelength limit X -> 2 u^2 (n13.H.n13 - n12.H.n12)
    # = 4 u^2 (A F+ (1 + cos^2 i)/2 + i A Fx cos i) up to a phase, so with cos i = 0,
    # <|X|^2> / (16 u^4 A^2) = 3/20, and with cos i = 1, <|X|^2> / (64 u^4 A^2) = <F+^2 + Fx^2> = 3/10.
    # A wrong tensor normalisation, basis or arm geometry moves these averages.
    g = np.random.default_rng(17)
    n = 6000
    f0, amp = 2e-6, 1e-22
    u = 2 * np.pi * f0 * C.L_ARM / C.C_LIGHT
    t = np.array([0.0])
    for cosi, scale, want in ((0.0, 16.0, 0.15), (1.0, 64.0, 0.30)):
        v = np.empty(n)
        for i in range(n):
            p = np.array([amp, f0, 0.0, 0.0, g.uniform(0, np.pi), cosi, g.uniform(-1, 1), g.uniform(0, 2 * np.pi)])
            X, _, _ = W.slow_tdi(p, t)
            v[i] = np.abs(X[0]) ** 2 / (scale * u ** 4 * amp ** 2)
        se = v.std() / np.sqrt(n)
        assert abs(v.mean() - want) < 5 * se + 2e-3 * want, (cosi, v.mean(), se)
