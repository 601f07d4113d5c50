"""The allocation-free total log-likelihood entry point.

Callers that cannot allocate device memory (code inside another framework's allocator
or memory budget, or that must not grow the device footprint) use
total_loglike_noalloc, whose only scratch is a fixed array inside the library. This
test calls it through the C ABI twice in a row, with different sizes, and checks each
result against total_loglike (which takes its scratch from a context) within the
tolerance the other likelihood tests use: float32 per-bin terms, |error| <= 3 n 2^-22;
then against the float64 oracle at 2^20 bins, twice in a row, to 5e-3 nats. It lives in a
file of its own that pytest collects last.
"""
import numpy as np
import pytest

from oracle import constants as OC
from paper_2405_04690_gb300 import synth

from _common import psd_window, torch_cuda

pytestmark = pytest.mark.gpu


def _residual(g, k0, n, psdp):
    nw = psdp.shape[0]
    r = np.empty((nw, 2, n), complex)
    for w in range(nw):
        s = psd_window(k0, n, psdp[w, 0], psdp[w, 1])
        r[w] = synth.unit_complex_normal(g, (2, n)) * np.sqrt(s / (4 * OC.DF))
    return r.astype(np.complex64)


def test_noalloc_total_loglike_matches_context_path_twice():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    dev = torch.device("cuda")
    g = synth.rng(31)
    cap = L.lib().total_loglike_noalloc_capacity()
    assert cap > 0
    for k0, n, nw in ((3146, 50001, 11), (40000, 20480, 5)):
        psdp = synth.draw_psd_params(g, nw)
        r = _residual(g, k0, n, psdp)
        rt = torch.from_numpy(r).view(torch.float32).reshape(nw, 2, n, 2).contiguous().to(dev)
        pt = torch.from_numpy(psdp).to(dev)
        want = torch.empty(nw, dtype=torch.float64, device=dev)
        got = torch.full((nw,), float("nan"), dtype=torch.float64, device=dev)
        ctx = L.Context(OC.TOBS, OC.DT, k0, n)
        L.total_loglike(ctx, rt, pt, want)
        L.total_loglike_noalloc(OC.TOBS, k0, n, rt, pt, got)
        torch.cuda.synchronize()
        w_np, g_np = want.cpu().numpy(), got.cpu().numpy()
        tol = 3 * n * 2.0 ** -22
        assert np.all(np.isfinite(g_np))
        assert np.max(np.abs(g_np - w_np)) < tol, (np.max(np.abs(g_np - w_np)), tol)
        ctx.close()


def test_noalloc_total_loglike_matches_oracle_at_a_million_bins():
    # The full-size window (k0 = 3146, 2^20 bins) against the float64 oracle's Eq. like, with
    # residuals whose noise level is off their walker's PSD by up to 30 %, so that a
    # systematic error of the PSD (of ln S or of 1/S) does not cancel between the two terms.
    torch = torch_cuda()
    from oracle import likelihood as LK
    from oracle import psd as OP
    from paper_2405_04690_gb300 import _lib as L
    dev = torch.device("cuda")
    g = synth.rng(32)
    k0, n, nw = 3146, 1 << 20, 3
    psdp = synth.draw_psd_params(g, nw)
    f = (k0 + np.arange(n)) / OC.TOBS
    r = np.empty((nw, 2, n), np.complex64)
    want = np.empty(nw)
    for w, scale in enumerate((0.7, 1.0, 1.3)):
        s = OP.psd_ae(f, psdp[w, 0], psdp[w, 1])
        r[w] = (scale * synth.unit_complex_normal(g, (2, n)) * np.sqrt(s / (4 * OC.DF))).astype(np.complex64)
        want[w] = LK.loglike(r[w].astype(np.complex128), s, OC.DF)
    rt = torch.from_numpy(r).view(torch.float32).reshape(nw, 2, n, 2).contiguous().to(dev)
    got = torch.full((nw,), float("nan"), dtype=torch.float64, device=dev)
    for _ in range(2):   # twice in a row: the shared scratch keeps the first call's contents
        L.total_loglike_noalloc(OC.TOBS, k0, n, rt, torch.from_numpy(psdp).to(dev), got)
        torch.cuda.synchronize()
        err = np.abs(got.cpu().numpy() - want)
        assert np.max(err) < 5e-3, (err, want)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    # correctly sized inputs that still exceed what the fixed array or the launch grid takes:
    # the call must refuse them with GBK_ERANGE before any kernel runs
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    dev = torch.device("cuda")
    cap = L.lib().total_loglike_noalloc_capacity()
    n = cap + 1                                     # the shape tables alone exceed the array
    tobs = 4 * OC.TOBS                              # keeps 3146 + n bins below f = c / (2L)
    r = torch.zeros((1, 2, n, 2), dtype=torch.float32, device=dev)
    pt = torch.ones((1, 2), dtype=torch.float64, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(L.GbkError) as ei:
        L.total_loglike_noalloc(tobs, 3146, n, r, pt, out)
    assert ei.value.status == 2
    nw = 65535 * 4 + 1                              # one walker more than the launch grid holds
    r = torch.zeros((nw, 2, 1, 2), dtype=torch.float32, device=dev)
    pt = torch.ones((nw, 2), dtype=torch.float64, device=dev)
    out = torch.zeros(nw, dtype=torch.float64, device=dev)
    with pytest.raises(L.GbkError) as ei:
        L.total_loglike_noalloc(OC.TOBS, 3146, 1, r, pt, out)
    assert ei.value.status == 2
