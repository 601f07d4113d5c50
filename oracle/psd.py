"""Noise PSD of the TDI A and E channels (test infrastructure).

Follows Sec. III of arXiv:2405.04690: Eq. psd

    S_n(x) = 8 sin^2(x) [ 2 S_pm (3 + 2 cos x + cos 2x) + S_op (2 + cos x) ],
    x = 2 pi f / f*,  f* = c / L,

with S_pm(f) = S_acc (2 pi c f)^-2 [1 + (0.4 mHz / f)^2] [1 + (f / 8 mHz)^4] and
S_op(f) = S_oms (2 pi f / c)^2 [1 + (2 mHz / f)^4]; and the Galactic foreground of
Sec. III.A, S_fg = 6 x^2 sin^2(x) h_fg(f) with
h_fg = (A_fg / 2) f^(-7/3) exp(-s1 f^alpha) [1 + tanh(-s2 (f - f_k))], added to S_n.

The model parameters are the amplitudes sqrt(S_oms) and sqrt(S_acc), as the paper
fits them (Sec. III, after Eq. psd). A and E share one PSD when one pair is given.
"""
import numpy as np

from .constants import C_LIGHT, L_ARM


def s_pm(f, sqrt_s_acc):
    """Acceleration-noise term S_pm(f) (Sec. III, the S_pm equation)."""
    f = np.asarray(f, dtype=np.float64)
    s_acc = sqrt_s_acc ** 2
    return (s_acc * (2.0 * np.pi * C_LIGHT * f) ** -2
            * (1.0 + (0.4e-3 / f) ** 2) * (1.0 + (f / 8e-3) ** 4))


def s_op(f, sqrt_s_oms):
    """Optical-metrology term S_op(f) (Sec. III, the S_op equation)."""
    f = np.asarray(f, dtype=np.float64)
    s_oms = sqrt_s_oms ** 2
    return s_oms * (2.0 * np.pi * f / C_LIGHT) ** 2 * (1.0 + (2e-3 / f) ** 4)


def psd_ae(f, sqrt_s_oms, sqrt_s_acc):
    """Instrument PSD of the A and E channels, Eq. psd."""
    f = np.asarray(f, dtype=np.float64)
    x = 2.0 * np.pi * f * L_ARM / C_LIGHT
    return 8.0 * np.sin(x) ** 2 * (2.0 * s_pm(f, sqrt_s_acc) * (3.0 + 2.0 * np.cos(x) + np.cos(2.0 * x))
                                   + s_op(f, sqrt_s_oms) * (2.0 + np.cos(x)))


def foreground_ae(f, a_fg, alpha, f_knee, s1, s2):
    """Galactic-foreground contribution S_fg to the A/E PSD (Sec. III.A)."""
    f = np.asarray(f, dtype=np.float64)
    x = 2.0 * np.pi * f * L_ARM / C_LIGHT
    h_fg = 0.5 * a_fg * f ** (-7.0 / 3.0) * np.exp(-s1 * f ** alpha) * (1.0 + np.tanh(-s2 * (f - f_knee)))
    return 6.0 * x ** 2 * np.sin(x) ** 2 * h_fg
