"""Uneven band lengths (N = 128..1024 by octave over 0.3-20 mHz) in one batch: per-N error
table against the oracle; the binned, autotuned launches give bit-identical results to a
single ragged launch (which, for its 1024-bin maximum, generates every waveform with a whole
block, the binned 128- and 256-bin launches with one warp: the two generators must give the
same bits); and the binned launches captured in one CUDA graph and replayed give the same bits
again."""
import numpy as np
import pytest

from oracle import constants as OC
from oracle import likelihood as OL
from oracle import residual as OR
from oracle import waveform as OW
from paper_2405_04690_gb300 import synth

from _common import FRAC_BITS, noise_fixed, psd_window, torch_cuda, window

pytestmark = pytest.mark.gpu


def _band_for(f0):
    return np.where(f0 < 1e-3, 128, np.where(f0 < 2e-3, 256, np.where(f0 < 4e-3, 512, 1024))).astype(np.int32)


def test_uneven_bands_error_table_and_binned_equals_ragged():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    dev = torch.device("cuda")
    g = synth.rng(41)
    n = 96
    p = synth.draw_sources(g, n, 3e-4, 2e-2, log_f=True)
    new = synth.perturb(g, p, synth.proposal_widths(p))
    nb = _band_for(p[1])
    k0, nbins = window(2.5e-4, 2.05e-2, 1100)
    s = psd_window(k0, nbins)
    rfix = noise_fixed(g, k0, nbins, s)
    r = OR.from_fixed(rfix, FRAC_BITS)
    want = np.array([OL.delta_loglike_swap(r, s, OC.DF, k0, OW.fastslow_band(new[:, i], int(nb[i])),
                                           OW.fastslow_band(p[:, i], int(nb[i]))) for i in range(n)])
    ctx = L.Context(OC.TOBS, OC.DT, k0, nbins)
    R = torch.from_numpy(rfix[None].copy()).to(dev)
    RS = L.residual_struct(R, FRAC_BITS)
    psdp = torch.tensor([[OC.SQRT_S_OMS, OC.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    PS = L.psd_struct(psdp)
    # one ragged launch
    out = torch.empty(n, dtype=torch.float64, device=dev)
    L.gb_delta_loglike_batch(ctx, torch.from_numpy(new).to(dev), torch.from_numpy(p).to(dev),
                             torch.from_numpy(nb).to(dev), 1024, torch.zeros(n, dtype=torch.int32, device=dev), RS, PS,
                             out, L.GBK_MIXED)
    L.gbk_sync_status(ctx)
    ragged = out.cpu().numpy()
    table = {}
    bins = {}
    for N in (128, 256, 512, 1024):
        idx = np.nonzero(nb == N)[0]
        if len(idx) == 0:
            continue
        err = np.abs(ragged[idx] - want[idx])
        table[N] = (len(idx), float(err.max()))
        assert err.max() < 1e-2, (N, err.max())
        # binned launch with an autotuned shape: bit-identical to the ragged launch
        pn = torch.from_numpy(np.ascontiguousarray(new[:, idx])).to(dev)
        po = torch.from_numpy(np.ascontiguousarray(p[:, idx])).to(dev)
        nbt = torch.full((len(idx),), N, dtype=torch.int32, device=dev)
        wt = torch.zeros(len(idx), dtype=torch.int32, device=dev)
        o2 = torch.empty(len(idx), dtype=torch.float64, device=dev)
        L.gbk_autotune_dlogl(ctx, pn, po, nbt, N, wt, RS, PS, o2, L.GBK_MIXED)
        L.gb_delta_loglike_batch(ctx, pn, po, nbt, N, wt, RS, PS, o2, L.GBK_MIXED)
        L.gbk_sync_status(ctx)
        assert np.array_equal(o2.cpu().numpy(), ragged[idx]), N
        bins[N] = (pn, po, nbt, wt, torch.full_like(o2, float("nan")))
    assert len(table) == 4, table
    print("per-N |Delta lnL error| (count, max):", table)
    # the four binned launches captured in one CUDA graph, replayed twice
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            for N, (pn, po, nbt, wt, o3) in bins.items():
                L.gb_delta_loglike_batch(ctx, pn, po, nbt, N, wt, RS, PS, o3, L.GBK_MIXED)
    torch.cuda.current_stream().wait_stream(cap)
    for _ in range(2):
        for o3 in (x[4] for x in bins.values()):
            o3.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        L.gbk_sync_status(ctx)
        for N, (_, _, _, _, o3) in bins.items():
            assert np.array_equal(o3.cpu().numpy(), ragged[np.nonzero(nb == N)[0]]), N
    ctx.close()
