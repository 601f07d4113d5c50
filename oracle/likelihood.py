"""Inner products and (Delta) log-likelihoods, FP64 (test infrastructure).

Follows Sec. II of arXiv:2405.04690:

* Eq. inner: <b|c> = 4 Re sum_f b~*(f) c~(f) / S_n(f) Delta f, summed here over the
  positive-frequency bins given and over the A and E channels.
* Eq. like: ln L = -1/2 <d - H | d - H> - sum_f ln S_n(f)  (both channels).
* Eq. addsource: Delta ln L_{+1} = -1/2 [<a|a> - 2 <d - H|a>].
* Eq. swapsource: Delta ln L_{+1/-1} = -1/2 [<a|a> + <r|r> - 2<a|r> - 2<d-H|a> + 2<d-H|r>].

Arrays of frequency-domain data have shape [2][n] (channel A, E; bins of a window
that starts at absolute bin k0). Bands are (k_start, A_band, E_band) triples.
"""
import numpy as np


def inner(b, c, psd, df):
    """Eq. inner over both channels; b, c complex [2][n], psd [n] or [2][n]."""
    b = np.asarray(b)
    c = np.asarray(c)
    psd = np.broadcast_to(np.asarray(psd, dtype=np.float64), b.shape)
    return 4.0 * df * float(np.sum(np.real(np.conj(b) * c) / psd))


def loglike(resid, psd, df):
    """Eq. like for a residual d - H given on a window of bins (both channels)."""
    psd = np.broadcast_to(np.asarray(psd, dtype=np.float64), np.shape(resid))
    return -0.5 * inner(resid, resid, psd, df) - float(np.sum(np.log(psd)))


def place(band, k0, n):
    """Put a band (k_start, A, E) into a zero window of n bins starting at bin k0."""
    k_start, a, e = band
    off = int(k_start) - int(k0)
    if off < 0 or off + len(a) > n:
        raise ValueError("band [%d, %d) outside window [%d, %d)" % (k_start, k_start + len(a), k0, k0 + n))
    w = np.zeros((2, n), dtype=np.complex128)
    w[0, off:off + len(a)] = a
    w[1, off:off + len(e)] = e
    return w


def delta_loglike_swap(resid, psd, df, k0, band_new, band_old):
    """Eq. swapsource: swap template r (band_old) for a (band_new) given d - H = resid.

    ``resid`` is the current residual d - H on the window starting at k0, with H
    including r. Either band may be None (then that template is zero): band_old=None
    gives Eq. addsource (a birth), band_new=None a removal.
    """
    n = np.shape(resid)[1]
    a = place(band_new, k0, n) if band_new is not None else np.zeros((2, n), complex)
    r = place(band_old, k0, n) if band_old is not None else np.zeros((2, n), complex)
    return -0.5 * (inner(a, a, psd, df) + inner(r, r, psd, df) - 2.0 * inner(a, r, psd, df)
                   - 2.0 * inner(resid, a, psd, df) + 2.0 * inner(resid, r, psd, df))


def delta_loglike_difference(resid, psd, df, k0, band_new, band_old):
    """Eq. swapsource regrouped as -1/2 <D|D> + <d-H|D>, D = a - r (same value).

    This is the algebraically identical grouping the GPU path evaluates; it is kept
    here only so a test can check it equals the expanded equation.
    """
    n = np.shape(resid)[1]
    a = place(band_new, k0, n) if band_new is not None else np.zeros((2, n), complex)
    r = place(band_old, k0, n) if band_old is not None else np.zeros((2, n), complex)
    d = a - r
    return -0.5 * inner(d, d, psd, df) + inner(resid, d, psd, df)


def delta_loglike_bruteforce(resid, psd, df, k0, band_new, band_old):
    """Difference of two full-window Eq. like evaluations (residual before/after)."""
    n = np.shape(resid)[1]
    a = place(band_new, k0, n) if band_new is not None else np.zeros((2, n), complex)
    r = place(band_old, k0, n) if band_old is not None else np.zeros((2, n), complex)
    after = resid - a + r
    return loglike(after, psd, df) - loglike(resid, psd, df)


def snr_optimal(band, psd, df, k0, n):
    """Optimal SNR sqrt(<h|h>) (Sec. II, after Eq. like)."""
    h = place(band, k0, n)
    return float(np.sqrt(inner(h, h, psd, df)))
