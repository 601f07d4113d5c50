"""What the trained learned proposal gains over the plain prior proposal.

A small ensemble (2 temperatures x 8 walkers, 6 bands, 2 loud sources per band in noise):
(1) sweeps from a near-truth start with the prior proposal; the cold chain's sources and
their band windows become training pairs; (2) the network is trained on them with the
library's kernels; (3) from an EMPTY model (no sources, residual = data) the sampler runs
the same number of sweeps with the prior proposal and with the learned one, same seeds.
The learned proposal must recover several times more of the injected sources in the same
number of sweeps; both runs keep the exact acceptance rule, so the learned one changes
only how fast the chain gets there.
"""
import math

import numpy as np
import pytest

from _common import torch_cuda
from _sweep_setup import FRAC, NB, key64, small_ensemble

pytestmark = pytest.mark.gpu

ALL = 1 | 2 | 4


def _recovered(cfg, truth_params, P, E):
    """Cold-chain sources within a bin in f0 and 0.3 in ln A of an injected source, per walker."""
    n = 0
    for w in range(cfg.n_walkers):
        for b in range(cfg.n_bands):
            for th in truth_params[b]:
                for bb in (b - 1, b, b + 1):
                    if not 0 <= bb < cfg.n_bands:
                        continue
                    ok = E[0, w, bb] & (np.abs(P[0, w, bb, :, 1] - th[1]) * cfg.tobs < 1.0) & \
                        (np.abs(np.log(np.maximum(P[0, w, bb, :, 0], 1e-30) / th[0])) < 0.3)
                    if ok.any():
                        n += 1
                        break
    return n


def test_trained_proposal_finds_sources_faster_than_the_prior():
    torch = torch_cuda()
    from paper_2405_04690_gb300 import _lib as L
    from paper_2405_04690_gb300 import proposal as PR
    from paper_2405_04690_gb300 import synth
    cfg, state, dfix, _ = small_ensemble(seed=20, n_temps=2, n_walkers=8, n_bands=6, n_max=6, n_per_band=2,
                                         betas=(1.0, 0.5))
    truth = [[state["params"][0, 0, b, i] for i in range(2)] for b in range(cfg.n_bands)]   # walker 0 ~ truth
    dev = torch.device("cuda")
    ctx = L.Context(cfg.tobs, 15.0, cfg.k0, cfg.n_bins)
    plan = L.SweepPlan(ctx, cfg.n_temps, cfg.n_walkers, cfg.n_bands, cfg.n_max, NB, cfg.band_k0, cfg.sigma,
                       L.GBK_MIXED, f_min=cfg.f_min, f_max=cfg.f_max)
    betas = torch.from_numpy(np.ascontiguousarray(cfg.betas)).to(dev)
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    PS = L.psd_struct(psdp)
    # (1) training pairs from the cold chain near the truth
    P = torch.from_numpy(state["params"].copy()).to(dev)
    E = torch.from_numpy(state["exists"].astype(np.uint8)).to(dev)
    R = torch.from_numpy(state["resid"].copy()).to(dev)
    RS = L.residual_struct(R, FRAC)
    buf = PR.PairBuffer(20000)
    for k in range(60):
        L.gb_sweep(plan, P, E, betas, RS, PS, key64(cfg), k, ALL | (L.SWEEP_REFRESH if k == 0 else 0))
        if k >= 10:
            buf.add_from_sweep(plan, P, E, RS, PS)
    assert buf.n > 4000
    # (2) training
    net = L.Mdn(512)
    tr = PR.Trainer(net, torch.from_numpy(PR.init_params(3)).to(dev), lr=1e-3)
    l_start = tr.mean_loss(buf, batch=512)
    for ep in range(40):
        tr.epoch(buf, 256, seed=100 + ep)
    l_end = tr.mean_loss(buf, batch=512)
    assert l_end < l_start - 10.0, (l_start, l_end)
    # (3) search from an empty model: prior proposal vs learned proposal
    results = {}
    for mode in ("prior", "learned"):
        P = torch.zeros_like(P)
        E = torch.zeros_like(E)
        R = torch.from_numpy(np.stack([dfix] * cfg.n_walkers)).to(dev).contiguous()
        RS = L.residual_struct(R, FRAC)
        stats = torch.zeros((5, 2), dtype=torch.int64, device=dev)
        flags = ALL
        if mode == "learned":
            L.gbk_sweep_set_proposal(plan, net=net, eps=0.2, inmodel_frac=0.25)
            flags |= L.SWEEP_MDN
        else:
            L.gbk_sweep_set_proposal(plan)
        curve = []
        for k in range(12):
            L.gb_sweep(plan, P, E, betas, RS, PS, key64(cfg) + 1, 1000 + k,
                       flags | (L.SWEEP_REFRESH if k == 0 else 0), stats=stats)
            curve.append(_recovered(cfg, truth, P.cpu().numpy(), E.cpu().numpy().astype(bool)))
        L.gbk_sync_status(ctx)
        results[mode] = (curve, stats.cpu().numpy())
    n_truth = cfg.n_walkers * cfg.n_bands * 2
    cp, sp = results["prior"]
    cl, sl = results["learned"]
    print("recovered of %d: prior %s, learned %s" % (n_truth, cp, cl))
    print("birth acceptance: prior %.4f learned %.4f" % (sp[1, 1] / sp[1, 0], sl[1, 1] / sl[1, 0]))
    print("training loss %.3f -> %.3f" % (l_start, l_end))
    assert cl[-1] >= 0.3 * n_truth and cl[-1] > 5 * max(cp[-1], 1)
    assert sum(cl) > 5 * max(sum(cp), 1)
    plan.close()
    ctx.close()
    net.close()
