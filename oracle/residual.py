"""Fixed-point residual d - H with a bit-exact add/subtract (test infrastructure).

The paper keeps a residual on the GPU and adds and removes template waveforms from it
(Alg. 1: r' <- r' + h(theta_k), r' <- r' - h(theta_k'); Alg. 2 likewise). Removing a
template that was added must give back the residual exactly (the inject-then-subtract
invariant); floating-point sums do not guarantee that, so the residual is held as
int64 fixed point: value = integer * 2^-frac_bits, each waveform value rounded to that
grid (round half to even) before the integer add or subtract.
"""
import numpy as np


def to_fixed(x, frac_bits):
    """Round complex values to the 2^-frac_bits grid; returns int64 [..., 2] (re, im)."""
    x = np.asarray(x, dtype=np.complex128)
    scale = np.ldexp(1.0, frac_bits)
    out = np.empty(x.shape + (2,), dtype=np.int64)
    out[..., 0] = np.rint(x.real * scale).astype(np.int64)
    out[..., 1] = np.rint(x.imag * scale).astype(np.int64)
    return out


def from_fixed(r, frac_bits):
    """Complex FP64 values of an int64 [..., 2] fixed-point array."""
    r = np.asarray(r, dtype=np.int64)
    return np.ldexp(r[..., 0].astype(np.float64), -frac_bits) + 1j * np.ldexp(r[..., 1].astype(np.float64), -frac_bits)


def add_sub(resid, k0, band, sign, frac_bits):
    """Add (sign=+1, the template enters the model: R -= h) or remove (sign=-1: R += h).

    ``resid`` is int64 [2][n][2] on the window starting at bin k0; returns a new array.
    """
    k_start, a, e = band
    off = int(k_start) - int(k0)
    n = resid.shape[1]
    if off < 0 or off + len(a) > n:
        raise ValueError("band outside residual window")
    out = np.array(resid, dtype=np.int64, copy=True)
    h = to_fixed(np.stack([a, e]), frac_bits)
    if sign > 0:
        out[:, off:off + len(a)] -= h
    else:
        out[:, off:off + len(a)] += h
    return out
