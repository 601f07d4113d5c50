"""Pins of the oracle's noise PSD (Eq. psd) and Galactic foreground (Sec. III.A)."""
import json
import os

import numpy as np

from oracle import constants as C
from oracle import psd as P
from oracle import likelihood as LK
from paper_2405_04690_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
FSTAR = C.C_LIGHT / C.L_ARM


def test_psd_zeros_at_multiples_of_pi():
    # Eq. psd carries 8 sin^2(x): the A/E response vanishes at x = k pi, f = k f*/2.
    for k in (1, 2, 3):
        f = k * FSTAR / 2.0
        s = P.psd_ae(np.array([f]), C.SQRT_S_OMS, C.SQRT_S_ACC)[0]
        s_near = P.psd_ae(np.array([f * 1.01]), C.SQRT_S_OMS, C.SQRT_S_ACC)[0]
        assert abs(s) < 1e-24 * abs(s_near)


def test_psd_low_frequency_limit():
    # x -> 0: sin^2 x -> x^2, 3 + 2cos x + cos 2x -> 6, 2 + cos x -> 3, so
    # S_n -> 8 x^2 (12 S_pm + 3 S_op); relative correction O(x^2).
    for f in (1e-5, 3e-5):
        x = 2 * np.pi * f / FSTAR
        lim = 8 * x * x * (12 * P.s_pm(f, C.SQRT_S_ACC) + 3 * P.s_op(f, C.SQRT_S_OMS))
        s = P.psd_ae(np.array([f]), C.SQRT_S_OMS, C.SQRT_S_ACC)[0]
        assert abs(s / lim - 1) < 2 * x * x


def test_psd_linear_in_noise_powers():
    f = np.geomspace(1e-4, 3e-2, 50)
    s_both = P.psd_ae(f, C.SQRT_S_OMS, C.SQRT_S_ACC)
    s_oms = P.psd_ae(f, C.SQRT_S_OMS, 0.0)
    s_acc = P.psd_ae(f, 0.0, C.SQRT_S_ACC)
    np.testing.assert_allclose(s_both, s_oms + s_acc, rtol=1e-13)
    np.testing.assert_allclose(P.psd_ae(f, 2 * C.SQRT_S_OMS, 0.0), 4 * s_oms, rtol=1e-13)
    assert np.all(s_both > 0)


def test_psd_shaping_knees():
    # The shaping factors equal 2 exactly at their knee frequencies.
    s_acc = C.SQRT_S_ACC ** 2
    for f, expect in ((0.4e-3, 2.0 * (1 + (0.4e-3 / 8e-3) ** 4)), (8e-3, 2.0 * (1 + (0.4e-3 / 8e-3) ** 2))):
        ratio = P.s_pm(f, C.SQRT_S_ACC) / (s_acc * (2 * np.pi * C.C_LIGHT * f) ** -2)
        assert abs(ratio / expect - 1) < 1e-13
    ratio = P.s_op(2e-3, C.SQRT_S_OMS) / (C.SQRT_S_OMS ** 2 * (2 * np.pi * 2e-3 / C.C_LIGHT) ** 2)
    assert abs(ratio - 2.0) < 1e-13


def test_foreground_crossing_matches_paper_statement():
    # Sec. VI.D: with the LDC2A instrument noise, the confusion foreground exceeds the
    # instrument PSD at ~1 mHz and drops below it around 4 mHz (Sec. III.A example).
    fg = GOLDEN["foreground_example"]
    nz = GOLDEN["ldc2a_noise"]
    st = GOLDEN["foreground_statement"]
    f = np.geomspace(5e-4, 1e-2, 2000)
    r = P.foreground_ae(f, fg["a_fg"], fg["alpha"], fg["f_knee"], fg["s1"], fg["s2"]) / P.psd_ae(f, nz["sqrt_s_oms"], nz["sqrt_s_acc"])
    at_1mhz = np.interp(st["above_psd_at_hz"], f, r)
    assert at_1mhz > 1.0
    crossing = f[np.where((r[:-1] > 1) & (r[1:] <= 1))[0][-1]]
    assert 0.6 * st["falls_below_near_hz"] < crossing < 1.4 * st["falls_below_near_hz"]


def test_noise_inner_product_chi2():
    # Noise with Re, Im ~ N(0, S/(4 df)) gives <n|n> ~ chi^2 with 2n d.o.f. per channel:
    # mean 2 per bin per channel (Eq. inner), checked to 5 sigma.
    g = synth.rng(7)
    k0, n = 31457, 40000
    f = (k0 + np.arange(n)) * C.DF
    s = P.psd_ae(f, C.SQRT_S_OMS, C.SQRT_S_ACC)
    z = synth.unit_complex_normal(g, (2, n)) * np.sqrt(s / (4 * C.DF))
    nn = LK.inner(z, z, s, C.DF)
    dof = 2 * 2 * n
    # <n|n> = sum of dof unit-variance squares
    assert abs(nn - dof) < 5 * np.sqrt(2 * dof)
