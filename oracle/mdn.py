"""Mixture-density-network proposal, float64 (test infrastructure).

The paper proposes births from Gaussian mixtures fitted to sampler output (Sec. V.E,
App. G) and names normalizing flows as future work (App. G); the learned proposal here is
a small MLP mixture density network. Its density must be exact for the Metropolis-Hastings
ratio of Eq. rj-acceptance, so it is a truncated diagonal Gaussian mixture on the unit box
in the coordinates where the band's prior is uniform:

    u0 = (ln A - ln A_min) / (ln A_max - ln A_min)     u1 = (f0 - lo_b) / (hi_b - lo_b)
    u2 = (Mc(f0, fdot) - mc_min) / (mc_max - mc_min)    u3 = phi0 / 2pi   u4 = psi / pi
    u5 = (cos i + 1) / 2   u6 = (sin b + 1) / 2   u7 = lambda / 2pi

(lo_b, hi_b the band's f0 allowance). In these coordinates the prior density is 1, so a
birth's Eq. rj-acceptance ratio is L^beta / q(u).

The proposal the sampler uses is the defensive mixture q(u) = eps + (1 - eps) q_MDN(u) (a
fraction eps of the draws come from the prior), so that no region of the prior is left
without proposals however the network was trained.

Network: 1024 whitened inputs -> 512 -> 512 -> 512 (ReLU) -> 272 = 16 x (1 logit + 8 mu
logits + 8 log-sigma logits); mu = sigmoid, ln sigma = S_MIN + (S_MAX - S_MIN) sigmoid,
mixture weights softmax. Weights are [out][in] matrices.
"""
import math

import numpy as np
from scipy.special import ndtr, ndtri

from . import philox as PX
from .constants import GM_SUN_C3

K_CHIRP = 96.0 / 5.0 * math.pi ** (8.0 / 3.0)

N_IN, N_HID, N_COMP, N_DIM = 1024, 512, 16, 8
N_OUT = N_COMP * (1 + 2 * N_DIM)
S_MIN, S_MAX = -10.0, 0.0
LAYERS = [(N_HID, N_IN), (N_HID, N_HID), (N_HID, N_HID), (N_OUT, N_HID)]
LOG_SQRT_2PI = 0.5 * math.log(2.0 * math.pi)


def n_params():
    return sum(o * i + o for o, i in LAYERS)


def unpack(theta):
    """Flat parameter vector -> list of (W [out][in], b [out]) in layer order."""
    out, k = [], 0
    for o, i in LAYERS:
        w = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((w, b))
    return out


# ---------------------------------------------------------------- coordinates
def to_unit(cfg, b, th):
    """Source parameters -> u in the unit box of band b (prior uniform)."""
    lo, hi = cfg.allowance(b)
    mc = (th[2] / (K_CHIRP * th[1] ** (11.0 / 3.0))) ** 0.6 / GM_SUN_C3
    return np.array([(math.log(th[0]) - cfg.ln_a_min) / (cfg.ln_a_max - cfg.ln_a_min), (th[1] - lo) / (hi - lo),
                     (mc - cfg.mc_min) / (cfg.mc_max - cfg.mc_min), th[3] / (2 * math.pi), th[4] / math.pi,
                     (th[5] + 1) / 2, (th[6] + 1) / 2, th[7] / (2 * math.pi)])


def from_unit(cfg, b, u):
    lo, hi = cfg.allowance(b)
    f0 = lo + (hi - lo) * u[1]
    mc = cfg.mc_min + (cfg.mc_max - cfg.mc_min) * u[2]
    return [math.exp(cfg.ln_a_min + (cfg.ln_a_max - cfg.ln_a_min) * u[0]), f0,
            K_CHIRP * f0 ** (11.0 / 3.0) * (mc * GM_SUN_C3) ** (5.0 / 3.0), 2 * math.pi * u[3], math.pi * u[4],
            2 * u[5] - 1, 2 * u[6] - 1, 2 * math.pi * u[7]]


# ---------------------------------------------------------------- network
def forward(theta, x, quantized=False):
    """x [B][1024] -> (raw outputs [B][272], cache of activations).

    quantized: the network as the tensor-core path defines it, with every weight matrix
    and every hidden activation rounded to bfloat16 (biases and outputs unrounded); the
    arithmetic between the rounding points stays float64."""
    layers = unpack(theta)
    acts = [x]
    h = x
    for li, (w, b) in enumerate(layers):
        z = h @ (to_bf16(w) if quantized else w).T + b
        if li < len(layers) - 1:
            h = np.maximum(z, 0.0)
            if quantized:
                h = to_bf16(h)
        else:
            h = z
        acts.append(h)
    return h, acts


def mixture(raw):
    """Raw outputs [B][272] -> (log pi [B][K], mu [B][K][8], log sigma [B][K][8])."""
    raw = raw.reshape(raw.shape[0], N_COMP, 1 + 2 * N_DIM)
    lg = raw[:, :, 0]
    lpi = lg - (np.log(np.sum(np.exp(lg - lg.max(axis=1, keepdims=True)), axis=1, keepdims=True))
                + lg.max(axis=1, keepdims=True))
    mu = 1.0 / (1.0 + np.exp(-raw[:, :, 1:1 + N_DIM]))
    ls = S_MIN + (S_MAX - S_MIN) / (1.0 + np.exp(-raw[:, :, 1 + N_DIM:]))
    return lpi, mu, ls


def log_trunc_normal(u, mu, ls):
    """ln of the normal density on [0, 1] renormalised by its mass there."""
    s = np.exp(ls)
    a, b = (1.0 - mu) / s, -mu / s
    logz = np.log(ndtr(a) - ndtr(b))
    return -0.5 * ((u - mu) / s) ** 2 - ls - LOG_SQRT_2PI - logz


def log_q(raw, u):
    """ln q(u) of the truncated diagonal mixture; raw [B][272], u [B][8]."""
    lpi, mu, ls = mixture(raw)
    comp = lpi + np.sum(log_trunc_normal(u[:, None, :], mu, ls), axis=2)
    m = comp.max(axis=1, keepdims=True)
    return (m + np.log(np.sum(np.exp(comp - m), axis=1, keepdims=True)))[:, 0]


def nll(theta, x, u):
    raw, _ = forward(theta, x)
    return -np.mean(log_q(raw, u))


def grad_raw(raw, u):
    """d(-ln q)/d raw for every sample (not averaged): [B][272]."""
    lpi, mu, ls = mixture(raw)
    s = np.exp(ls)
    a, bb = (1.0 - mu) / s, -mu / s
    z = ndtr(a) - ndtr(bb)
    pa, pb = np.exp(-0.5 * a * a) / math.sqrt(2 * math.pi), np.exp(-0.5 * bb * bb) / math.sqrt(2 * math.pi)
    lt = -0.5 * ((u[:, None, :] - mu) / s) ** 2 - ls - LOG_SQRT_2PI - np.log(z)
    comp = lpi + lt.sum(axis=2)
    m = comp.max(axis=1, keepdims=True)
    lq = m + np.log(np.sum(np.exp(comp - m), axis=1, keepdims=True))
    r = np.exp(comp - lq)                                   # responsibilities
    pi = np.exp(lpi)
    d = np.zeros((raw.shape[0], N_COMP, 1 + 2 * N_DIM))
    d[:, :, 0] = pi - r
    dlt_dmu = (u[:, None, :] - mu) / s ** 2 - (pb - pa) / (s * z)
    dlt_dls = ((u[:, None, :] - mu) / s) ** 2 - 1.0 - (-a * pa + bb * pb) / z
    d[:, :, 1:1 + N_DIM] = -r[:, :, None] * dlt_dmu * mu * (1 - mu)
    sg = (ls - S_MIN) / (S_MAX - S_MIN)
    d[:, :, 1 + N_DIM:] = -r[:, :, None] * dlt_dls * (S_MAX - S_MIN) * sg * (1 - sg)
    return d.reshape(raw.shape[0], -1)


def backward(theta, x, u, quantized=False):
    """Gradient of the mean NLL with respect to the flat parameters (quantized: of the
    bfloat16-rounded network of ``forward``, rounding passed through as the identity)."""
    layers = unpack(theta)
    if quantized:
        layers = [(to_bf16(w), b) for w, b in layers]
    raw, acts = forward(theta, x, quantized)
    g = grad_raw(raw, u) / x.shape[0]
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        w, _ = layers[li]
        h_in = acts[li]
        gw = g.T @ h_in
        gb = g.sum(axis=0)
        grads.append((gw, gb))
        if li > 0:
            g = (g @ w) * (acts[li] > 0)
    out = []
    for gw, gb in reversed(grads):
        out.append(gw.ravel())
        out.append(gb)
    return np.concatenate(out)


def adam(theta, m, v, grad, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on float64 arrays; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def sample(raw, g):
    """Draw u from the truncated mixture for each row of raw (inverse CDF per dimension)."""
    lpi, mu, ls = mixture(raw)
    out = np.empty((raw.shape[0], N_DIM))
    for i in range(raw.shape[0]):
        k = g.choice(N_COMP, p=np.exp(lpi[i]) / np.exp(lpi[i]).sum())
        s = np.exp(ls[i, k])
        lo, hi = ndtr(-mu[i, k] / s), ndtr((1 - mu[i, k]) / s)
        out[i] = np.clip(mu[i, k] + s * ndtri(lo + (hi - lo) * g.uniform(size=N_DIM)), 0.0, 1.0)
    return out


def init_params(g, scale=1.0, out_scale=0.1, width_bias=2.0):
    """He-style random initialisation (for tests and as a training start): hidden layers
    N(0, 2 / fan_in) x scale, the output layer a further x out_scale, and the width-logit
    biases at width_bias (s = e^(-10 + 10 sigmoid(2)) ~ 0.3: broad components to start)."""
    out = []
    for li, (o, i) in enumerate(LAYERS):
        sc = scale * (out_scale if li == len(LAYERS) - 1 else 1.0)
        out.append((g.standard_normal((o, i)) * sc * math.sqrt(2.0 / i)).ravel())
        b = np.zeros(o)
        if li == len(LAYERS) - 1:
            b.reshape(N_COMP, 1 + 2 * N_DIM)[:, 1 + N_DIM:] = width_bias
        out.append(b)
    return np.concatenate(out)


# ---------------------------------------------------------------- inputs
def to_bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), via float32."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def features(rho, psd_w, df, nb=256):
    """Whitened residual of a band's own sub-band: x[ch 512 + 2 i + {0: Re, 1: Im}] =
    rho[ch][nb + i] sqrt(4 df / S_n), i < nb, rho the band window [2][3 nb] (sub-bands b-1, b,
    b+1) with the band's own sources added back, psd_w the PSD on the window. Noise-only bins
    are standard normal in each of Re and Im (Eq. inner's weight 4 df / S_n)."""
    c = rho[:, nb:2 * nb] * np.sqrt(4.0 * df / psd_w[nb:2 * nb])[None, :]
    x = np.empty(4 * nb)
    for ch in range(2):
        x[ch * 2 * nb:(ch + 1) * 2 * nb:2] = c[ch].real
        x[ch * 2 * nb + 1:(ch + 1) * 2 * nb:2] = c[ch].imag
    return x


# ---------------------------------------------------------------- proposal used by the sampler
def log_q_defensive(raw_row, u, eps):
    """ln[eps + (1 - eps) q_MDN(u)] for one mixture (raw_row [272]) at one point u [8]."""
    lq = float(log_q(np.asarray(raw_row)[None, :], np.asarray(u)[None, :])[0])
    if eps >= 1.0:
        return 0.0
    if eps <= 0.0:
        return lq
    return float(np.logaddexp(math.log(eps), math.log1p(-eps) + lq))


def draw_unit(raw_row, w_comp, w_dims):
    """u from the truncated mixture: component = first k whose cumulative weight exceeds
    u32(w_comp) (the last if rounding leaves none); per dimension the inverse CDF
    u_d = mu + s Phi^-1(Phi(-mu/s) + [Phi((1-mu)/s) - Phi(-mu/s)] u32(w_d)), clamped to [0, 1]."""
    lpi, mu, ls = mixture(np.asarray(raw_row)[None, :])
    pi = np.exp(lpi[0])
    v = PX.u32(w_comp)
    k, c = N_COMP - 1, 0.0
    for j in range(N_COMP):
        c += pi[j]
        if v < c:
            k = j
            break
    u = np.empty(N_DIM)
    for d in range(N_DIM):
        m, s = mu[0, k, d], math.exp(ls[0, k, d])
        lo, hi = ndtr(-m / s), ndtr((1.0 - m) / s)
        u[d] = min(max(m + s * ndtri(lo + (hi - lo) * PX.u32(w_dims[d])), 0.0), 1.0)
    return u
