"""Host-side pins of the float generator's shorter-series path (no GPU).

For a source with x = 2 pi f_max L/c <= 0.25 the float32 slow part cuts its small-argument
series short: exp(i y) after y^7 (sin) and y^8 (cos), sin(pi s)/(pi s) after (pi s)^6, and it
forms each link phase pi f L/c k.n_a - 2 pi f k.dx_j / c as one series of the summed argument.
These tests check what that rests on: the craft offsets from the guiding centre are L/sqrt3
in the orbit model, so no argument exceeds (1/2 + 1/sqrt3) x, and the dropped terms stay below
1e-10 relative over that range. The GPU parity of the path itself is in test_gpu_core.py.
"""
import math

import numpy as np

import bench
from oracle import constants as OC
from oracle import orbits as OO

X_MAX = 0.25                                   # limit on 2 pi f_max L/c
LINK_MAX = (0.5 + 1.0 / math.sqrt(3.0)) * X_MAX   # largest link-phase argument


def test_craft_offsets_from_the_guiding_centre_are_l_over_sqrt3():
    t = np.linspace(0.0, OC.YEAR, 2001)
    x = OO.spacecraft_positions(t)                # [craft][xyz][time]
    gc = x.mean(axis=0)
    d = np.sqrt(((x - gc[None]) ** 2).sum(axis=1)) / OC.L_ARM
    assert np.max(np.abs(d - 1.0 / math.sqrt(3.0))) < 1e-9
    # the guiding centre is the circular orbit the kernel's orbit table uses
    a = 2.0 * np.pi * t / OC.YEAR
    assert np.max(np.abs(gc[0] - OC.AU * np.cos(a))) < 1e-6 * OC.L_ARM
    assert np.max(np.abs(gc[2])) < 1e-6 * OC.L_ARM


def test_link_phase_arguments_stay_in_the_short_series_range():
    # |pi f L/c k.n| <= x/2 and |2 pi f k.dx/c| <= x/sqrt3 with |k| = |n| = 1, |dx| = L/sqrt3
    assert LINK_MAX < 0.27
    g = np.random.default_rng(3)
    k = g.standard_normal((3, 4000))
    k /= np.linalg.norm(k, axis=0)
    t = g.uniform(0.0, OC.YEAR, 4000)
    x = OO.spacecraft_positions(t)
    gc = x.mean(axis=0)
    n = OO.arm_unit(x[0], x[1])
    f = X_MAX / (2.0 * np.pi * OC.L_ARM / OC.C_LIGHT)
    lc = OC.L_ARM / OC.C_LIGHT
    for j in range(3):
        dx = (x[j] - gc) / OC.C_LIGHT
        arg = np.pi * f * lc * (k * n).sum(axis=0) - 2.0 * np.pi * f * (k * dx).sum(axis=0)
        assert np.max(np.abs(arg)) <= LINK_MAX * (1 + 1e-12)


def test_dropped_terms_are_below_1e_10():
    y = np.linspace(-0.27, 0.27, 20001)
    y = y[y != 0.0]
    z = y * y
    sin7 = y * (1.0 - z / 6.0 + z * z / 120.0 - z ** 3 / 5040.0)
    cos8 = 1.0 - z / 2.0 + z * z / 24.0 - z ** 3 / 720.0 + z ** 4 / 40320.0
    assert np.max(np.abs(sin7 - np.sin(y)) / np.abs(np.sin(y))) < 1e-10
    assert np.max(np.abs(cos8 - np.cos(y))) < 1e-10
    s = np.linspace(-X_MAX / np.pi, X_MAX / np.pi, 20001)
    s = s[s != 0.0]
    w = (np.pi * s) ** 2
    sinc6 = 1.0 - w / 6.0 + w * w / 120.0 - w ** 3 / 5040.0
    assert np.max(np.abs(sinc6 - np.sinc(s)) / np.abs(np.sinc(s))) < 1e-10


def test_bench_counts_the_short_series_below_4p77_mhz():
    f_lim = X_MAX / (2.0 * np.pi * OC.L_ARM / OC.C_LIGHT)
    assert 4.77e-3 < f_lim < 4.78e-3
    assert bench.short_series(f_lim * (1 - 1e-9)) and not bench.short_series(f_lim * (1 + 1e-9))
    assert bench.flops_per_waveform(256, True) == 256 * 477 + 2 * 5 * 256 * 8
    assert bench.flops_per_waveform(256) == 256 * 621 + 2 * 5 * 256 * 8
    # every source of the bench ensemble (1-4 mHz bands, allowance half a band above) is short
    f_top = (math.floor(bench.F_HI * bench.TOBS) + 1.5 * bench.N_BAND) / bench.TOBS + 1e-7
    assert bench.short_series(f_top)
