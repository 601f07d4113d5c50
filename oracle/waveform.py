"""Galactic-binary TDI A/E waveform, FP64 (test infrastructure).

The paper re-implements FastGB (Sec. II.A, App. F): a slow-part response on a coarse
time grid, an FFT of that slow part, and a heterodyne to the carrier bin; it prints no
formula for it. The oracle therefore gives the model in two forms:

* ``fastslow_band`` (W2) -- the fast/slow decomposition, what the GPU computes.
* ``bruteforce_tdi`` / ``bruteforce_band`` (W1) -- the same physical model evaluated
  exactly at every fine sample with a direct DFT; W2 is pinned against it.

Model (readings where the paper is silent):

* 8 parameters A, f0, fdot, phi0, psi, cos(iota), sin(beta), lambda.
* h_+ = A (1 + cos^2 iota) cos Phi, h_x = -2 A cos iota sin Phi,
  Phi(t) = phi0 + 2 pi f0 t + pi fdot t^2, so the complex strain tensor is
  Hc = A (1 + cos^2 iota) e_+(psi) + 2 i A cos(iota) e_x(psi) and H(t) = Re[Hc e^{i Phi}].
* Propagation direction k = -(cos b cos l, cos b sin l, sin b); polarisation basis
  u = (sin b cos l, sin b sin l, -cos b), v = (sin l, -cos l, 0), e_+ = uu - vv,
  e_x = uv + vu, rotated by psi: e_+(psi) = cos2psi e_+ - sin2psi e_x,
  e_x(psi) = sin2psi e_+ + cos2psi e_x.
* Link i->j received at time t (rigid equal arms of length L along the unit vector n
  from craft i to craft j; emitter at x_j - L n):
  y_ij(t) = n.H.n / (2 (1 - k.n)) [H(t - L/c - (k.x_j - L k.n)/c) - H(t - k.x_j/c)].
* First-generation Michelson X with equal constant arms (TDI 1.5 in Sec. II):
  X(t) = y31(t) + y13(t-L) + y21(t-2L) + y12(t-3L) - y21(t) - y12(t-L) - y31(t-2L) - y13(t-3L),
  Y and Z by the cyclic map 1->2->3->1; A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6
  (Sec. II, the A_1/E_1 definitions).
* DFT x~(f_k) = dt sum_n x(t_n) e^{-2 pi i k n / N_t}; the band of a source holds bins
  [q - N/2, q + N/2) with q = floor(f0 T).
"""
import numpy as np

from .constants import C_LIGHT, L_ARM, TOBS
from .orbits import spacecraft_positions, arm_unit

# (receiver-craft index pairs) for the six links, as (sender, receiver), 0-based.
LINKS = {"12": (0, 1), "21": (1, 0), "23": (1, 2), "32": (2, 1), "31": (2, 0), "13": (0, 2)}


def _geometry(params):
    """Propagation vector, polarisation basis and complex tensor amplitude of one source."""
    amp, f0, fdot, phi0, psi, cosi, sinb, lam = [float(v) for v in params]
    cosb = np.sqrt(1.0 - sinb * sinb)
    k = -np.array([cosb * np.cos(lam), cosb * np.sin(lam), sinb])
    u = np.array([sinb * np.cos(lam), sinb * np.sin(lam), -cosb])
    v = np.array([np.sin(lam), -np.cos(lam), 0.0])
    ep = np.outer(u, u) - np.outer(v, v)
    ex = np.outer(u, v) + np.outer(v, u)
    c2, s2 = np.cos(2.0 * psi), np.sin(2.0 * psi)
    ep_psi = c2 * ep - s2 * ex
    ex_psi = s2 * ep + c2 * ex
    hc = amp * (1.0 + cosi * cosi) * ep_psi + 2j * amp * cosi * ex_psi
    return k, hc


def _nhn(hc, n):
    """n.Hc.n for unit vectors n of shape [3][time]."""
    return np.einsum("it,ij,jt->t", n, hc, n)


def slow_tdi(params, t):
    """Slow parts X, Y, Z (complex, per sample) of the fast/slow decomposition.

    Uses the approximation Phi(t - tau) ~ Phi(t) - 2 pi f(t) tau with
    f(t) = f0 + fdot t, and all geometry (positions, arm vectors) at the sample time.
    Returns the factors multiplying e^{i Phi(t)}.
    """
    amp, f0, fdot = float(params[0]), float(params[1]), float(params[2])
    k, hc = _geometry(params)
    t = np.asarray(t, dtype=np.float64)
    x = spacecraft_positions(t)
    f = f0 + fdot * t
    lc = L_ARM / C_LIGHT
    y = {}
    for name, (i, j) in LINKS.items():
        n = arm_unit(x[i], x[j])
        kn = k @ n
        kxj = k @ x[j] / C_LIGHT
        half = np.pi * f * lc * (1.0 - kn)
        sinc = np.sinc(half / np.pi)                      # sin(half)/half
        y[name] = (_nhn(hc, n) * (-1j * np.pi * f * lc) * sinc * np.exp(-1j * half)
                   * np.exp(-2j * np.pi * f * kxj))
    d = np.exp(-2j * np.pi * f * lc)
    pre = 1.0 - d * d
    X = pre * ((y["31"] - y["21"]) + d * (y["13"] - y["12"]))
    Y = pre * ((y["12"] - y["32"]) + d * (y["21"] - y["23"]))
    Z = pre * ((y["23"] - y["13"]) + d * (y["32"] - y["31"]))
    return X, Y, Z


def carrier_bin(f0, tobs=TOBS):
    """q = floor(f0 T) and delta = f0 T - q."""
    ft = float(f0) * tobs
    q = int(np.floor(ft))
    return q, ft - q


def fastslow_band(params, n_band, tobs=TOBS):
    """W2: A and E over bins [q - N/2, q + N/2) by the fast/slow decomposition.

    Steps (App. F): slow part on N coarse samples t_p = p T / N; multiply by the
    heterodyned phase exp(i(phi0 + 2 pi delta p / N + pi fdot t_p^2)); N-point FFT;
    scale by T / (2 N) (the 1/2 takes the positive-frequency half of the real signal);
    place offset m in [-N/2, N/2) at bin q + m.
    Returns (k_start, A_band, E_band) with k_start = q - N/2.
    """
    amp, f0, fdot, phi0 = [float(v) for v in params[:4]]
    q, delta = carrier_bin(f0, tobs)
    p = np.arange(n_band, dtype=np.float64)
    t = p * tobs / n_band
    X, Y, Z = slow_tdi(params, t)
    a_slow = (Z - X) / np.sqrt(2.0)
    e_slow = (X - 2.0 * Y + Z) / np.sqrt(6.0)
    het = np.exp(1j * (phi0 + 2.0 * np.pi * delta * p / n_band + np.pi * fdot * t * t))
    scale = 0.5 * tobs / n_band
    m = np.arange(-n_band // 2, n_band // 2)
    a_fft = np.fft.fft(a_slow * het) * scale
    e_fft = np.fft.fft(e_slow * het) * scale
    return q - n_band // 2, a_fft[m % n_band], e_fft[m % n_band]


def bruteforce_tdi(params, t):
    """W1: complex analytic A and E at every time t, evaluating the model exactly.

    Each link is evaluated at the exact delayed time of each TDI term, with the exact
    phase Phi at the emission and reception events (no Taylor expansion) and the
    geometry at the delayed reception time.
    """
    amp, f0, fdot, phi0 = [float(v) for v in params[:4]]
    k, hc = _geometry(params)
    lc = L_ARM / C_LIGHT

    def phase(tt):
        return phi0 + 2.0 * np.pi * f0 * tt + np.pi * fdot * tt * tt

    t = np.asarray(t, dtype=np.float64)
    # geometry at the four delayed reception times t - m L/c, m = 0..3
    pos = {m: spacecraft_positions(t - m * lc) for m in range(4)}

    def link(name, m):
        i, j = LINKS[name]
        tr = t - m * lc
        x = pos[m]
        n = arm_unit(x[i], x[j])
        kn = k @ n
        kxj = k @ x[j] / C_LIGHT
        t_emit = tr - lc - (kxj - lc * kn)
        t_recv = tr - kxj
        return _nhn(hc, n) / (2.0 * (1.0 - kn)) * (np.exp(1j * phase(t_emit)) - np.exp(1j * phase(t_recv)))

    def michelson(a, b, c):
        # X-type combination read at craft a with arms to b and c; link names are
        # sender+receiver, the second argument the delay in units of L/c.
        return (link(c + a, 0) + link(a + c, 1) + link(b + a, 2) + link(a + b, 3)
                - link(b + a, 0) - link(a + b, 1) - link(c + a, 2) - link(a + c, 3))

    X = michelson("1", "2", "3")
    Y = michelson("2", "3", "1")
    Z = michelson("3", "1", "2")
    return (Z - X) / np.sqrt(2.0), (X - 2.0 * Y + Z) / np.sqrt(6.0)


def bruteforce_band(params, n_band, n_t, dt, fold=True):
    """W1 band: direct DFT of the fine-sampled analytic A/E signal, halved.

    With fold=True the DFT is summed over all bins congruent modulo N (the aliases of
    each band offset), which the N-point FFT of the fast/slow path reproduces exactly
    when N divides N_t; fold=False returns the plain DFT at bins q - N/2 .. q + N/2 - 1.
    """
    tobs = n_t * dt
    q, _ = carrier_bin(params[1], tobs)
    t = np.arange(n_t, dtype=np.float64) * dt
    za, ze = bruteforce_tdi(params, t)
    bins = q - n_band // 2 + np.arange(n_band)
    out = []
    for z in (za, ze):
        spec = np.fft.fft(z) * dt
        if fold:
            folded = spec.reshape(n_t // n_band, n_band).sum(axis=0)
            out.append(0.5 * folded[bins % n_band])
        else:
            out.append(0.5 * spec[bins % n_t])
    return q - n_band // 2, out[0], out[1]
