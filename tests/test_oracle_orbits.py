"""Pins of the oracle's analytic orbits (oracle/orbits.py), which the fast/slow waveform and its
brute-force check share (a mistake here would move both and pass their comparison): the
properties the paper's TDI 1.5 reading assumes (Sec. II: a rigid constellation with equal,
constant arms) and the closed-form geometry of first-order heliocentric orbits with e = L /
(2 sqrt(3) AU): centroid on the 1 AU circle, arms of length L at every time, constellation
plane at 60 degrees to the ecliptic, one-year period and one cartwheel turn per year."""
import math

import numpy as np

from oracle import constants as OC
from oracle import orbits as OO

T = np.linspace(0.0, OC.YEAR, 1201)


def test_centroid_follows_the_1_au_circle():
    x = OO.spacecraft_positions(T)
    cen = x.mean(axis=0)
    a = 2.0 * math.pi * T / OC.YEAR
    want = np.array([OC.AU * np.cos(a), OC.AU * np.sin(a), np.zeros_like(a)])
    assert np.abs(cen - want).max() < 1e-12 * OC.AU


def test_arms_are_equal_and_constant():
    x = OO.spacecraft_positions(T)
    for i, j in ((0, 1), (1, 2), (2, 0)):
        d = np.linalg.norm(x[i] - x[j], axis=0)
        assert np.abs(d / OC.L_ARM - 1.0).max() < 1e-12, (i, j)


def test_constellation_plane_is_inclined_60_degrees():
    # the normal makes 60 degrees with the ecliptic pole and leans 30 degrees out of the plane
    # through the Sun: n . r_hat = -cos(30 deg) (first-order orbits keep this exactly)
    x = OO.spacecraft_positions(T)
    n = np.cross((x[1] - x[0]).T, (x[2] - x[0]).T)
    n /= np.linalg.norm(n, axis=1)[:, None]
    assert np.abs(np.abs(n[:, 2]) - 0.5).max() < 1e-12
    cen = x.mean(axis=0).T
    r = cen / np.linalg.norm(cen, axis=1)[:, None]
    assert np.abs(np.abs((n * r).sum(axis=1)) - math.sqrt(3.0) / 2.0).max() < 1e-12


def test_one_year_period_and_unit_arms():
    x0 = OO.spacecraft_positions(np.array([0.0, 1.0e6]))
    x1 = OO.spacecraft_positions(np.array([OC.YEAR, OC.YEAR + 1.0e6]))
    assert np.abs(x1 - x0).max() < 1e-12 * OC.AU
    x = OO.spacecraft_positions(T)
    for i, j in ((0, 1), (1, 2), (2, 0)):
        nij = OO.arm_unit(x[i], x[j])
        assert np.abs(np.linalg.norm(nij, axis=0) - 1.0).max() < 1e-14
        assert np.array_equal(OO.arm_unit(x[j], x[i]), -nij)
    # the cartwheel: in the plane spanned by u1 = -(r_hat + sqrt3 z_hat)/2 and the direction of
    # motion phi_hat, craft n sits at angle alpha - 2 pi n / 3 on the circle of radius L / sqrt3
    # around the centroid (the circumradius of the equilateral triangle): one turn per year
    cen = x.mean(axis=0)
    a = 2.0 * math.pi * T / OC.YEAR
    r_hat = np.array([np.cos(a), np.sin(a), np.zeros_like(a)])
    phi_hat = np.array([-np.sin(a), np.cos(a), np.zeros_like(a)])
    for n in range(3):
        d = x[n] - cen
        c1 = -0.5 * (np.sum(d * r_hat, axis=0) + math.sqrt(3.0) * d[2])
        c2 = np.sum(d * phi_hat, axis=0)
        want = a - 2.0 * math.pi * n / 3.0
        rad = OC.L_ARM / math.sqrt(3.0)
        assert np.abs(c1 - rad * np.cos(want)).max() < 1e-9 * rad
        assert np.abs(c2 - rad * np.sin(want)).max() < 1e-9 * rad
        assert np.abs(np.linalg.norm(d, axis=0) / rad - 1.0).max() < 1e-12
