"""Batched Gaussian-mixture refit on the GPU (gmm_fit) against the float64 oracle (oracle/gmm.py).

Six groups on the same seeded inputs: separated clusters with absent (NaN) rows, an empty
group, fewer points than components, points without mixture structure, clusters with
repeated rows and tied f0 values, and a dense three-cluster group. FP64: weights, means and
variances to 1e-9 (EM from the same start for the same iterations; the two sides differ only
in summation order), log-likelihoods to 1e-10, mixture outputs to float32 rounding. Mixed
(float32 E-step, sums centred on the current means): with one component per cluster, where
EM is well conditioned, means to 1e-4 of their widths, variances to 1e-4 and weights to 1e-6
(float32 rounding of responsibilities and centred terms, ~1e-7, with margin); with 16
components, where components share clusters and EM is ill conditioned, the log-likelihood
of the fit to 1e-3 nats per point.
"""
import numpy as np
import pytest

from oracle import gmm as GM

from _common import torch_cuda

pytestmark = pytest.mark.gpu

P = 600


def _groups():
    g = np.random.default_rng(11)
    x = np.full((6, P, 8), np.nan)

    def clusters(k, n_each, sig):
        c = g.uniform(0.15, 0.85, (k, 8))
        return np.concatenate([c[j] + sig[j] * g.standard_normal((n_each, 8)) for j in range(k)])

    a = clusters(4, 140, [0.01, 0.02, 0.005, 0.015])
    x[0, :560] = a[g.permutation(560)]
    x[0, g.choice(560, 25, replace=False)] = np.nan            # absent rows among the present
    x[2, [3, 50, 51, 300, 599]] = g.uniform(0, 1, (5, 8))      # 5 points < 16 components
    x[3] = g.uniform(0, 1, (P, 8))                              # no structure
    b = clusters(3, 100, [0.01, 0.01, 0.02])
    x[4, :300] = b
    x[4, 300:400] = b[:100]                                     # repeated rows
    x[4, 400:420, 1] = x[4, 0, 1]                               # tied f0 values
    x[4, 400:420, [0, 2, 3, 4, 5, 6, 7]] = 0.5
    x[5] = clusters(3, 200, [0.003, 0.01, 0.03])
    return x.astype(np.float32)


def _oracle(x, n_iter):
    out = []
    for grp in x.astype(np.float64):
        w, mu, var, hist = GM.fit(grp, n_iter=n_iter)
        out.append((w, mu, var, hist[-1] if hist else 0.0, GM.to_raw(w, mu, var)))
    return out


def _gpu(torch, x, n_iter, precision):
    from paper_2405_04690_gb300 import _lib as L
    xt = torch.from_numpy(x).cuda()
    raw = torch.full((2, x.shape[0], 272), np.nan, dtype=torch.float32, device="cuda")
    fit = torch.zeros((x.shape[0], 16, 17), dtype=torch.float64, device="cuda")
    ll = torch.zeros(x.shape[0], dtype=torch.float64, device="cuda")
    L.gmm_fit(xt, raw, n_iter=n_iter, precision=precision, fit_out=fit, loglike=ll)
    torch.cuda.synchronize()
    raw = raw.cpu().numpy()
    assert np.array_equal(raw[0], raw[1])   # n_copies
    return raw[0], fit.cpu().numpy(), ll.cpu().numpy()


@pytest.mark.parametrize("n_iter", [0, 30])
def test_gmm_fit_fp64_matches_oracle(n_iter):
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    x = _groups()
    want = _oracle(x, n_iter)
    raw, fit, ll = _gpu(torch, x, n_iter, L.GBK_FP64)
    for gi, (w, mu, var, lw, rw) in enumerate(want):
        k = len(w)
        np.testing.assert_allclose(fit[gi, :k, 0], w, rtol=1e-9, atol=1e-14, err_msg=str(gi))
        np.testing.assert_allclose(fit[gi, :k, 1:9], mu, rtol=1e-9, atol=1e-12, err_msg=str(gi))
        np.testing.assert_allclose(fit[gi, :k, 9:], var, rtol=1e-9, atol=1e-15, err_msg=str(gi))
        assert (fit[gi, k:] == 0).all()
        assert abs(ll[gi] - lw) <= 1e-10 * max(1.0, abs(lw)), (gi, ll[gi], lw)
        np.testing.assert_allclose(raw[gi], rw.astype(np.float32), rtol=1e-6, atol=1e-6, err_msg=str(gi))
    assert len(want[1][0]) == 0 and len(want[2][0]) == 5


def test_gmm_fit_mixed_matches_oracle_on_clusters():
    # one component per cluster (well-conditioned EM): parameters to the stated tolerances
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    x = _groups()
    for groups, k in (((0,), 4), ((4, 5), 3)):
        xs = np.ascontiguousarray(x[list(groups)])
        want = [GM.fit(grp, n_comp=k, n_iter=40) for grp in xs.astype(np.float64)]
        xt = torch.from_numpy(xs).cuda()
        raw = torch.empty((1, len(groups), 272), dtype=torch.float32, device="cuda")
        fit = torch.zeros((len(groups), 16, 17), dtype=torch.float64, device="cuda")
        L.gmm_fit(xt, raw, n_comp=k, n_iter=40, precision=L.GBK_MIXED, fit_out=fit)
        fit = fit.cpu().numpy()
        for i, (w, mu, var, _) in enumerate(want):
            sig = np.sqrt(var)
            assert np.abs(fit[i, :k, 0] - w).max() < 1e-6, groups[i]
            assert (np.abs(fit[i, :k, 1:9] - mu) / sig).max() < 1e-4, groups[i]
            assert (np.abs(fit[i, :k, 9:] - var) / var).max() < 1e-4, groups[i]


def test_gmm_fit_mixed_likelihood_with_16_components():
    # 16 components on 3-4 clusters: several components share a cluster and EM trades weight
    # among them slowly, so float32 rounding sends the iteration along a slightly different
    # path (individual weights move by ~1e-5, and the log-likelihood reached differs by ~2e-4
    # nats per point, up or down); the fitted density stays within 1e-3 nats per point
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    x = _groups()
    want = _oracle(x, 40)
    raw, fit, ll = _gpu(torch, x, 40, L.GBK_MIXED)
    for gi in (0, 2, 3, 4, 5):
        lw = want[gi][3]
        n = int((~np.isnan(x[gi]).any(axis=1)).sum())
        assert abs(ll[gi] - lw) < 1e-3 * n, (gi, ll[gi], lw)
    assert np.isfinite(raw).all()


def test_gmm_fit_uses_the_first_present_rows_up_to_the_cap():
    # 3000 rows (100 absent) of three clusters in one group: the library fits the first
    # gmm_max_points() present rows, as the oracle does with the same cap (FP64, 1e-9)
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    cap = L.gmm_max_points()
    g = np.random.default_rng(12)
    c = g.uniform(0.2, 0.8, (3, 8))
    x = np.concatenate([c[j] + 0.01 * g.standard_normal((1000, 8)) for j in range(3)])
    x[g.choice(3000, 100, replace=False)] = np.nan
    x = x.astype(np.float32)[None]
    assert (~np.isnan(x[0]).any(axis=1)).sum() > cap
    w, mu, var, hist = GM.fit(x[0].astype(np.float64), n_iter=20, cap=cap)
    raw = torch.empty((1, 1, 272), dtype=torch.float32, device="cuda")
    fit = torch.zeros((1, 16, 17), dtype=torch.float64, device="cuda")
    ll = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.gmm_fit(torch.from_numpy(x).cuda(), raw, n_iter=20, precision=L.GBK_FP64, fit_out=fit, loglike=ll)
    fit = fit.cpu().numpy()[0]
    np.testing.assert_allclose(fit[:, 0], w, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(fit[:, 1:9], mu, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(fit[:, 9:], var, rtol=1e-9, atol=1e-15)
    assert abs(ll.item() - hist[-1]) <= 1e-10 * abs(hist[-1])
