"""Analytic LISA orbits for the oracle (test infrastructure).

The paper assumes a rigid constellation with equal, constant arms for TDI 1.5
(Sec. II, below Eq. swapsource) and names no orbit model. Reading: the
standard first-order-in-eccentricity heliocentric orbits, orbital phase and
constellation orientation both zero at t = 0,

    alpha(t) = 2 pi t / year,   beta_n = 2 pi (n - 1) / 3,   e = L / (2 sqrt(3) AU)
    x_n = AU cos(alpha) + (e AU / 2) [cos(2 alpha - beta_n) - 3 cos(beta_n)]
    y_n = AU sin(alpha) + (e AU / 2) [sin(2 alpha - beta_n) - 3 sin(beta_n)]
    z_n = -sqrt(3) e AU cos(alpha - beta_n)

for spacecraft n = 1, 2, 3. Arm unit vectors point from sender to receiver.
"""
import numpy as np

from .constants import AU, L_ARM, YEAR


def spacecraft_positions(t):
    """Positions of the three spacecraft, shape (3, 3, len(t)) = [craft][xyz][time], m."""
    t = np.asarray(t, dtype=np.float64)
    ecc = L_ARM / (2.0 * np.sqrt(3.0) * AU)
    alpha = 2.0 * np.pi * t / YEAR
    out = np.empty((3, 3) + t.shape, dtype=np.float64)
    for n in range(3):
        beta_n = 2.0 * np.pi * n / 3.0
        out[n, 0] = AU * np.cos(alpha) + 0.5 * ecc * AU * (np.cos(2 * alpha - beta_n) - 3 * np.cos(beta_n))
        out[n, 1] = AU * np.sin(alpha) + 0.5 * ecc * AU * (np.sin(2 * alpha - beta_n) - 3 * np.sin(beta_n))
        out[n, 2] = -np.sqrt(3.0) * ecc * AU * np.cos(alpha - beta_n)
    return out


def arm_unit(x_from, x_to):
    """Unit vector from one spacecraft position array [xyz][time] to another."""
    d = x_to - x_from
    return d / np.sqrt(np.sum(d * d, axis=0))
