"""The ensemble sweep at the benchmark's full size and launch configuration (16 temperatures x 32
walkers x 369 sub-bands, 2000 injected sources, mixed precision, one step = sweep + ownership
transfer), checked through properties that hold at any size and on sampled windows against
the float64 oracle.

1. Exact bookkeeping: after two steps, every walker's cold residual equals the data minus the
   walker's final cold sources, rebuilt from scratch with the library's own templates (int64
   fixed point, so bit for bit): no accepted change was lost or applied twice anywhere.
2. Independent waveforms on sampled windows: for 24 random (walker, sub-band) windows, the final
   residual plus the oracle's float64 templates of the walker's final cold sources, minus the
   oracle's templates of the injected sources, gives back the injected noise to the float32
   template error (1e-5 of the summed template norms; the mixed waveform's error is ~4e-7 each).
3. The move statistics add up: every proposal is counted once, acceptances never exceed them.
"""
import os
import sys

import numpy as np
import pytest

from oracle import residual as OR
from oracle import waveform as OW

from _common import torch_cuda

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_full_size_sweep_bookkeeping_and_sampled_windows():
    torch = torch_cuda()
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as BN
    from paper_2405_04690_gb300 import _lib as L
    dev = torch.device("cuda")
    ens = BN.build_ensemble(seed=1, n_temps=BN.N_T)
    S = BN.build_device_state(torch, L, dev, ens, L.GBK_MIXED, seed=1)
    P0 = S["P"].clone()
    E0 = S["E"].clone()
    R0 = S["resid"].clone()
    stats = torch.zeros((5, 2), dtype=torch.int64, device=dev)
    xfer = torch.zeros(2, dtype=torch.int32, device=dev)
    for k in range(2):
        L.gb_sweep(S["plan"], S["P"], S["E"], S["betas"], S["R"], S["psd"], 0xF011, k,
                   1 | 2 | 4 | (L.SWEEP_REFRESH if k == 0 else 0), stats=stats)
        L.gbk_sweep_transfer(S["plan"], S["P"], S["E"], xfer)
    L.gbk_sync_status(S["ctx"])
    nw, nb_ = BN.N_W, BN.N_BAND
    # (1) rebuild every walker's residual: data = R0 + initial cold templates; expected = data - final cold
    chk = R0.clone()
    RC = L.residual_struct(chk, BN.FRAC_BITS)

    def move(P, E, sign):
        cold = P[0].reshape(-1, 8)[E[0].reshape(-1).bool()]
        wv = E[0].reshape(nw, -1).bool().nonzero()[:, 0].to(torch.int32)
        L.residual_add_sub(S["ctx"], RC, cold.t().contiguous(), torch.full((cold.shape[0],), nb_, dtype=torch.int32,
                           device=dev), nb_, wv, sign, L.GBK_MIXED)

    move(P0, E0, -1)
    move(S["P"], S["E"], +1)
    L.gbk_sync_status(S["ctx"])
    assert torch.equal(chk, S["resid"]), int((chk != S["resid"]).sum().item())
    # (3) statistics
    st = stats.cpu().numpy()
    assert (st[:4, 1] <= st[:4, 0]).all() and st[:4, 0].sum() > 9e6 and xfer[0].item() > 0
    # (2) sampled windows against the oracle's float64 templates
    g = np.random.default_rng(4)
    P = S["P"].cpu().numpy()
    E = S["E"].cpu().numpy().astype(bool)
    R = S["resid"].cpu().numpy()
    noise = OR.from_fixed(S["noise"].cpu().numpy(), BN.FRAC_BITS)
    truth = ens["truth"]
    tobs, k0 = BN.TOBS, ens["k0"]
    worst = 0.0
    for _ in range(24):
        w = int(g.integers(nw))
        b = int(g.integers(1, ens["n_bands"] - 1))
        lo = ens["band_k0"] + (b - 1) * nb_ - k0
        hi = lo + 3 * nb_
        got = OR.from_fixed(R[w], BN.FRAC_BITS)[:, lo:hi]
        acc = np.zeros((2, hi - lo), complex)
        norm = 0.0
        srcs = [(P[0, w][E[0, w]].reshape(-1, 8), +1.0), (truth.T, -1.0)]
        for arr, sign in srcs:
            for th in arr:
                q = int(np.floor(th[1] * tobs)) - k0
                if q + nb_ // 2 <= lo or q - nb_ // 2 >= hi:
                    continue
                ks, a, e = OW.fastslow_band(th, nb_, tobs)
                o = ks - k0 - lo
                i0, i1 = max(0, o), min(hi - lo, o + nb_)
                acc[0, i0:i1] += sign * a[i0 - o:i1 - o]
                acc[1, i0:i1] += sign * e[i0 - o:i1 - o]
                norm += np.linalg.norm(np.concatenate([a, e]))
        diff = got + acc - noise[:, lo:hi]
        rel = np.linalg.norm(diff) / max(norm, 1e-300)
        worst = max(worst, rel)
    assert worst < 1e-5, worst
    S["plan"].close()
    S["ctx"].close()
