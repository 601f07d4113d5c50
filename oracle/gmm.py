"""Gaussian-mixture refit proposal, float64 (test infrastructure).

Sec. V.E and App. G: besides the prior, the paper proposes reversible-jump births from
Gaussian mixture models fitted to samples (the cold chain's recent sources for the "refit"
proposal, a per-band search's samples for the "search" proposal), fitted with scikit-learn
on CPUs, each fitted group then given equal probability in one larger mixture; it names
batched GPU fitting as the desirable form. Here every band's recent cold-chain sources are
fitted in the band's unit coordinates (``oracle.mdn.to_unit``: the prior is uniform on the
unit box there) by expectation-maximisation (Dempster, Laird & Rubin 1977) for a
diagonal-covariance mixture:

    E-step   r_ik = w_k N(x_i; mu_k, var_k) / sum_j w_j N(x_i; mu_j, var_j)
    M-step   N_k = sum_i r_ik,  w_k = N_k / sum_j N_j,  mu_k = sum_i r_ik x_i / N_k,
             var_k = sum_i r_ik (x_i - mu_k)^2 / N_k + reg

Readings (the paper gives no fitting details): diagonal covariances, so that the fitted
mixture is the truncated diagonal family the sampler already evaluates exactly; K = min(16,
n) components; start: the present points sorted by u1 (f0; ties by position), initial means
the points of rank floor((k + 1/2) n / K), initial variances the group's per-dimension
variance + reg, weights 1 / K; a fixed number of EM iterations; reg = 1e-6 (scikit-learn's
default reg_covar). The paper's equal probability per fitted group becomes equal weights
for the components that hold at least ``min_weight`` of the band's points (the others keep
a weight of e^-30 relative); the result is written as the 272 mixture outputs (``raw``)
that ``oracle.mdn.mixture`` reads: weight logits, logit(mu), logit((ln sigma - S_MIN) /
(S_MAX - S_MIN)), clamped into the open intervals.

Pinned in tests/test_oracle_gmm.py against scikit-learn's GaussianMixture (same start,
same iterations), the EM monotonicity of the log-likelihood, recovery of separated clusters
and a worked initialisation example.
"""
import math

import numpy as np

from .mdn import N_COMP, N_DIM, S_MAX, S_MIN

LOG_2PI = math.log(2.0 * math.pi)
W_OFF = -30.0          # weight logit of a component left out of the proposal
CLAMP = 1e-9           # open-interval clamp of the logits


def present(x):
    """Rows of x [P][8] without NaN, in order."""
    x = np.asarray(x, dtype=np.float64)
    return x[~np.isnan(x).any(axis=1)]


def init(x, n_comp=N_COMP, reg=1e-6):
    """Start of EM for the present points x [n][8]: (w [K], mu [K][8], var [K][8])."""
    n = x.shape[0]
    k = min(n_comp, n)
    order = np.argsort(x[:, 1], kind="stable")
    mu = np.array([x[order[int(math.floor((j + 0.5) * n / k))]] for j in range(k)])
    var = np.tile(x.var(axis=0) + reg, (k, 1))
    return np.full(k, 1.0 / k), mu, var


def log_density(x, w, mu, var):
    """ln w_k + ln N(x_i; mu_k, var_k) for every point and component: [n][K]."""
    d = x[:, None, :] - mu[None, :, :]
    return np.log(w)[None, :] - 0.5 * np.sum(d * d / var[None, :, :] + np.log(var)[None, :, :] + LOG_2PI, axis=2)


def e_step(x, w, mu, var):
    """Responsibilities [n][K] and the total log-likelihood sum_i ln sum_k w_k N_ik."""
    lp = log_density(x, w, mu, var)
    m = lp.max(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(np.exp(lp - m).sum(axis=1))
    return np.exp(lp - lse[:, None]), float(lse.sum())


def m_step(x, r, reg=1e-6):
    """N_k carries scikit-learn's 10 eps guard (a component that lost every point keeps finite
    parameters: mean 0, variance reg, weight ~1e-15 / n); weights normalised by sum N_k."""
    nk = r.sum(axis=0) + 10.0 * np.finfo(np.float64).eps
    mu = (r.T @ x) / nk[:, None]
    var = np.stack([(r[:, j:j + 1] * (x - mu[j]) ** 2).sum(axis=0) / nk[j] for j in range(r.shape[1])]) + reg
    return nk / nk.sum(), mu, var


def fit(x, n_comp=N_COMP, n_iter=50, reg=1e-6, cap=None):
    """EM from ``init``: n_iter (E, M) iterations on the present rows (the first ``cap`` of them
    when given). Returns (w, mu, var, history) with history the log-likelihood before each
    M-step and, last, that of the returned parameters."""
    x = present(x)
    if cap is not None:
        x = x[:cap]
    if x.shape[0] == 0:
        return np.zeros(0), np.zeros((0, N_DIM)), np.zeros((0, N_DIM)), []
    w, mu, var = init(x, n_comp, reg)
    hist = []
    for _ in range(n_iter):
        r, ll = e_step(x, w, mu, var)
        hist.append(ll)
        w, mu, var = m_step(x, r, reg)
    hist.append(e_step(x, w, mu, var)[1])
    return w, mu, var, hist


def _logit(p):
    p = min(max(p, CLAMP), 1.0 - CLAMP)
    return math.log(p / (1.0 - p))


def to_raw(w, mu, var, min_weight=0.01):
    """The fitted mixture as the sampler's 272 mixture outputs (16 x (logit, 8 mu, 8 sigma))."""
    raw = np.zeros((N_COMP, 1 + 2 * N_DIM))
    k = len(w)
    used = [j for j in range(k) if w[j] >= min_weight]
    if k and not used:
        used = [int(np.argmax(w))]
    for j in range(N_COMP):
        if j < k:
            raw[j, 0] = 0.0 if j in used else W_OFF
            for d in range(N_DIM):
                raw[j, 1 + d] = _logit(mu[j, d])
                raw[j, 1 + N_DIM + d] = _logit((0.5 * math.log(var[j, d]) - S_MIN) / (S_MAX - S_MIN))
        else:   # no points (or fewer than 16): broad components centred in the box
            raw[j, 0] = 0.0 if k == 0 else W_OFF
            raw[j, 1:1 + N_DIM] = 0.0
            raw[j, 1 + N_DIM:] = _logit(1.0)
    return raw.ravel()
