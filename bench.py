"""Benchmark of the GB sampler hot path on GB300 (one JSON line on stdout).

Workload (the batched ensemble): 16 temperatures x 32 walkers; the data are seeded noise
plus 2,000 Galactic binaries with f0 in 1-4 mHz (N = 256 band bins, 369 sub-bands);
every walker holds its own jittered copy of the 2,000 sources at every temperature
(1,024,000 sources), sorted into sub-band slots. One step is one full sweep of the
sampler (gb_sweep): odd then even sub-bands, each band with one in-model proposal per
source (Alg. 1), the flip-all reversible jump over its n_max slots (App. C) and the
ensemble-permuted tempering swaps (Alg. 2), with the cold-chain residual of every
walker on the device (int64 fixed point) updated in place. Mixed precision.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own replica of the workload (weak scaling); rank 0
prints the max-over-ranks timing.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_T, N_W, N_SRC, N_BAND = 16, 32, 2000, 256
FRAC_BITS = 98
TOBS = 2 ** 21 * 15.0
DT = 15.0
F_LO, F_HI = 1e-3, 4e-3
METRIC = "GB proposals (waveform+DeltalogL) /sec"
WORKLOAD = ("batched ensemble: 16 temps x 32 walkers x 2000 GBs (1-4 mHz, N=256, 369 sub-bands); one step = one "
            "full sweep (in-model 1/source + flip-all RJ + PT swaps), mixed precision")

# Algorithmic float32 work (counted from the operations of the method):
# slow-part response 621 flops per coarse sample, 477 for a source with 2 pi f_max L/c <= 0.25
# (f below 4.77 mHz: the generator then cuts its Taylor series short and forms each link
# phase from its summed argument), band FFT 5 N log2 N per channel, Delta lnL 45 flops per
# band bin.
FLOPS_SLOW_PER_SAMPLE = 621
FLOPS_SLOW_PER_SAMPLE_SHORT = 477
SHORT_SERIES_ARG = 0.25
L_OVER_C = 2.5e9 / 299792458.0
FLOPS_PER_BIN = 45


def short_series(f_max):
    """True where the generator takes the shorter series (f_max: the largest |f| of the source)."""
    return 2.0 * math.pi * f_max * L_OVER_C <= SHORT_SERIES_ARG


def f_max_of(p):
    """Largest |f| of each source ([8][n] parameters) over the observation."""
    return np.maximum(np.abs(p[1]), np.abs(p[1] + p[2] * TOBS))


def flops_per_waveform(n=N_BAND, short=False):
    per = FLOPS_SLOW_PER_SAMPLE_SHORT if short else FLOPS_SLOW_PER_SAMPLE
    return n * per + 2 * 5 * n * int(math.log2(n))


def flops_per_evaluation(n=N_BAND):
    return n * FLOPS_PER_BIN


PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
K_BAND_TRAFFIC = 8 * (1156.076e6 + 761.686e6)   # DRAM bytes per band-kernel launch (ncu, scaled)


def measured_hbm_gbs():
    """Measured copy bandwidth of the GB300s, else the profiling fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def autocorr_time(x, c=5.0):
    """Integrated autocorrelation time of series x [n_chains][n_steps] (mean ACF over
    chains, Sokal's adaptive window: smallest M with M >= c tau(M))."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[1]
    xc = x - x.mean(axis=1, keepdims=True)
    f = np.fft.rfft(xc, n=2 * n, axis=1)
    acf = np.fft.irfft(f * np.conj(f), axis=1)[:, :n]
    acf = acf / np.maximum(acf[:, :1], 1e-300)
    rho = acf.mean(axis=0)
    taus = 2.0 * np.cumsum(rho) - 1.0
    for m in range(1, n):
        if m >= c * taus[m]:
            return float(taus[m])
    return float(taus[-1])


# ------------------------------------------------------------------ CPU oracle timing
def _oracle_worker(args):
    seed, n_bands = args
    sys.path.insert(0, ROOT)
    from oracle import constants as OC
    from oracle import mcmc as OM
    from oracle import psd as OP
    from oracle import residual as OR
    from oracle import waveform as OW
    from paper_2405_04690_gb300 import synth
    g = synth.rng(seed)
    band_k0 = int(math.floor(2.0e-3 * OC.TOBS)) + 256 * (seed % 50)
    k0 = band_k0 - 2 * N_BAND
    n_bins = (n_bands + 4) * N_BAND
    f = (k0 + np.arange(n_bins)) * OC.DF
    s = OP.psd_ae(f, OC.SQRT_S_OMS, OC.SQRT_S_ACC)
    n_t, n_w, n_max = 2, 1, 8
    cfg = OM.SweepConfig(tobs=OC.TOBS, k0=k0, n_bins=n_bins, band_k0=band_k0, nb=N_BAND, n_bands=n_bands,
                         n_temps=n_t, n_walkers=n_w, n_max=n_max, betas=np.tile([1.0, 0.5], (n_bands, 1)),
                         psd=np.tile(s, (n_w, 1)), sigma=sweep_sigma(), key=(seed, 99))
    params = np.zeros((n_t, n_w, n_bands, n_max, 8))
    exists = np.zeros((n_t, n_w, n_bands, n_max), dtype=bool)
    data = synth.unit_complex_normal(g, (2, n_bins)) * np.sqrt(s / (4 * OC.DF))
    for b in range(n_bands):
        lo, hi = cfg.band_bins(b)
        p = synth.draw_sources(g, 5, (lo + 2) / OC.TOBS, (hi - 2) / OC.TOBS)
        params[:, :, b, :5] = p.T[None, None]
        exists[:, :, b, :5] = True
    r = OR.to_fixed(data, FRAC_BITS)
    for b in range(n_bands):
        for i in range(5):
            r = OR.add_sub(r, k0, OW.fastslow_band(params[0, 0, b, i], N_BAND), +1, FRAC_BITS)
    state = {"params": params, "exists": exists, "resid": r[None].copy()}
    t0 = time.perf_counter()
    trace = OM.sweep(cfg, state, 0)
    return time.perf_counter() - t0, len(trace)


def cpu_baseline(n_bands=48, cores=None):
    """Time the FP64 oracle sweep on a bounded sample over all host cores (spawned pool)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(7000 + i, n_bands) for i in range(cores)])
    wall = time.perf_counter() - t0
    done = sum(c for _, c in res)
    busy = max(t for t, _ in res)
    return {"value": done / busy, "unit": "proposals/s", "cores": cores, "kind": "oracle",
            "value_per_core": float(np.mean([c / t for t, c in res])),
            "sample": "%d proposals: %d processes each run one FP64 oracle sweep of 2 temps x 1 walker x %d sub-bands "
                      "(5 GBs/band, 8 slots) near 2 mHz; %.1f s wall incl. pool start" % (done, cores, n_bands, wall)}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ workload on the GPU
def sweep_sigma():
    df = 1.0 / TOBS
    return [0.05, 0.1 * df, 0.005 * df / TOBS, 0.05, 0.05, 0.02, 0.02, 0.02]


def ladder(n_temps):
    """Temperatures 1.2^t, the top one infinite (beta = 0)."""
    b = np.array([1.2 ** -t for t in range(n_temps)])
    b[-1] = 0.0
    return b


def build_ensemble(seed, n_temps=N_T, n_walkers=N_W, n_src=N_SRC):
    """Host arrays of the ensemble: params [T][W][B][n_max][8], exists, band layout."""
    from paper_2405_04690_gb300 import synth
    g = synth.rng(seed)
    band_k0 = int(math.floor(F_LO * TOBS))
    n_bands = int(math.ceil((math.floor(F_HI * TOBS) - band_k0) / N_BAND))
    truth = synth.draw_sources(g, n_src, F_LO, F_HI)
    band = ((np.floor(truth[1] * TOBS).astype(np.int64) - band_k0) // N_BAND).astype(np.int64)
    counts = np.bincount(band, minlength=n_bands)
    n_max = int(math.ceil(1.5 * counts.max()))
    slot = np.zeros(n_src, dtype=np.int64)
    seen = np.zeros(n_bands, dtype=np.int64)
    for i in np.argsort(band, kind="stable"):
        slot[i] = seen[band[i]]
        seen[band[i]] += 1
    params = np.zeros((n_temps, n_walkers, n_bands, n_max, 8))
    exists = np.zeros((n_temps, n_walkers, n_bands, n_max), dtype=np.uint8)
    df = 1.0 / TOBS
    jit = np.array([0.0, 0.02 * df, 0.0, 0.02, 0.02, 0.01, 0.01, 0.01])[:, None]
    for t in range(n_temps):
        for w in range(n_walkers):
            p = truth + jit * g.standard_normal(truth.shape)
            p[0] = truth[0] * np.exp(0.02 * g.standard_normal(n_src))
            p[5] = np.clip(p[5], -1, 1)
            p[6] = np.clip(p[6], -1, 1)
            p[3] %= 2 * np.pi
            p[4] %= np.pi
            p[7] %= 2 * np.pi
            params[t, w, band, slot] = p.T
            exists[t, w, band, slot] = 1
    return {"truth": truth, "params": params, "exists": exists, "band_k0": band_k0, "n_bands": n_bands,
            "n_max": n_max, "k0": band_k0 - 2 * N_BAND, "n_bins": (n_bands + 4) * N_BAND}


def build_device_state(torch, L, dev, ens, precision, seed):
    from paper_2405_04690_gb300 import synth
    g = synth.rng(seed + 17)
    nt, nw = ens["params"].shape[:2]
    ctx = L.Context(TOBS, DT, ens["k0"], ens["n_bins"])
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    s = torch.empty((1, ens["n_bins"]), dtype=torch.float64, device=dev)
    L.psd_eval(ctx, psdp, s)
    z = torch.from_numpy(synth.unit_complex_normal(g, (2, ens["n_bins"]))).to(dev)
    noise = z * torch.sqrt(s[0] * (TOBS / 4.0))
    scale = float(2.0 ** FRAC_BITS)
    one = torch.stack([torch.round(noise.real * scale), torch.round(noise.imag * scale)], dim=-1).to(torch.int64)
    resid = one.unsqueeze(0).repeat(nw, 1, 1, 1).contiguous()
    R = L.residual_struct(resid, FRAC_BITS)
    truth = ens["truth"]
    nsrc = truth.shape[1]
    nb = torch.full((nsrc,), N_BAND, dtype=torch.int32, device=dev)
    tt = torch.from_numpy(truth).to(dev)
    for w in range(nw):   # data = noise + injected sources (templates leave the model: R += h)
        L.residual_add_sub(ctx, R, tt, nb, N_BAND, torch.full((nsrc,), w, dtype=torch.int32, device=dev), -1, precision)
    P = torch.from_numpy(ens["params"]).to(dev)
    E = torch.from_numpy(ens["exists"]).to(dev)
    cold = ens["params"][0].reshape(-1, 8)[ens["exists"][0].reshape(-1).astype(bool)]
    wv = np.nonzero(ens["exists"][0])[0].astype(np.int32)
    L.residual_add_sub(ctx, R, torch.from_numpy(np.ascontiguousarray(cold.T)).to(dev),
                       torch.full((len(wv),), N_BAND, dtype=torch.int32, device=dev), N_BAND,
                       torch.from_numpy(wv).to(dev), +1, precision)
    betas = torch.from_numpy(np.tile(ladder(nt), (ens["n_bands"], 1))).to(dev).contiguous()
    plan = L.SweepPlan(ctx, nt, nw, ens["n_bands"], ens["n_max"], N_BAND, ens["band_k0"], sweep_sigma(), precision,
                       f_min=F_LO, f_max=F_HI)
    L.gbk_sync_status(ctx)
    return {"ctx": ctx, "plan": plan, "P": P, "E": E, "resid": resid, "R": R, "psd": L.psd_struct(psdp),
            "psdp": psdp, "betas": betas, "noise": one}


def band_for(f0):
    """Band length by octave: 128 below 1 mHz, doubling per octave up to 1024."""
    return np.where(f0 < 1e-3, 128, np.where(f0 < 2e-3, 256, np.where(f0 < 4e-3, 512, 1024))).astype(np.int32)


def run_uneven(torch, L, dev, stream, seed, n_prop=200000, reps=10):
    from paper_2405_04690_gb300 import synth
    g = synth.rng(seed)
    p = synth.draw_sources(g, n_prop, 3e-4, 2e-2, log_f=True)
    new = synth.perturb(g, p, synth.proposal_widths(p))
    nb = band_for(p[1])
    k0, nbins = synth.window_for(2.5e-4, 2.05e-2, 1100)
    ctx = L.Context(TOBS, DT, k0, nbins)
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    s = torch.empty((1, nbins), dtype=torch.float64, device=dev)
    L.psd_eval(ctx, psdp, s)
    z = torch.from_numpy(synth.unit_complex_normal(g, (2, nbins))).to(dev)
    noise = z * torch.sqrt(s[0] * (TOBS / 4.0))
    scale = float(2.0 ** FRAC_BITS)
    resid = torch.stack([torch.round(noise.real * scale), torch.round(noise.imag * scale)],
                        dim=-1).to(torch.int64).unsqueeze(0).contiguous()
    R = L.residual_struct(resid, FRAC_BITS)
    P = L.psd_struct(psdp)
    groups = {}
    for n in (128, 256, 512, 1024):
        idx = np.nonzero(nb == n)[0]
        if len(idx) == 0:
            continue
        m = len(idx)
        groups[n] = {"new": torch.from_numpy(np.ascontiguousarray(new[:, idx])).to(dev),
                     "old": torch.from_numpy(np.ascontiguousarray(p[:, idx])).to(dev),
                     "nb": torch.full((m,), n, dtype=torch.int32, device=dev),
                     "w": torch.zeros(m, dtype=torch.int32, device=dev),
                     "out": torch.empty(m, dtype=torch.float64, device=dev), "m": m,
                     # per proposal: both waveforms (each with its own series length) and one
                     # evaluation of N bins
                     "flops": sum(n_short * flops_per_waveform(n, True) + (m - n_short) * flops_per_waveform(n)
                                  for n_short in (int(short_series(f_max_of(new[:, idx])).sum()),
                                                  int(short_series(f_max_of(p[:, idx])).sum())))
                              + m * n * FLOPS_PER_BIN}
    per_n = {}
    for n, G in groups.items():
        best = L.gbk_autotune_dlogl(ctx, G["new"], G["old"], G["nb"], n, G["w"], R, P, G["out"], L.GBK_MIXED, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            L.gb_delta_loglike_batch(ctx, G["new"], G["old"], G["nb"], n, G["w"], R, P, G["out"], L.GBK_MIXED, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        per_n[str(n)] = {"proposals": G["m"], "proposals_per_s": G["m"] / (ms * 1e-3),
                         "waveforms_per_s": 2 * G["m"] / (ms * 1e-3), "tuned_warps_per_cta": best[0],
                         "tuned_ctas_per_sm": best[1] or "max",
                         "fp32_frac": G["flops"] / (ms * 1e-3) / 1e12 / PEAK_FP32_TFLOPS}
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            for n, G in groups.items():
                L.gb_delta_loglike_batch(ctx, G["new"], G["old"], G["nb"], n, G["w"], R, P, G["out"], L.GBK_MIXED)
    torch.cuda.current_stream().wait_stream(cap)
    graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    L.gbk_sync_status(ctx)
    ctx.close()
    return {"workload": "200,000 proposals, f0 log-uniform 0.3-20 mHz, N = 128/256/512/1024 by octave; binned by N, "
                        "autotuned launch shape per N, one CUDA graph of the 4 launches",
            "proposals_per_s": n_prop / (ms * 1e-3), "ms_per_batch": ms, "per_N": per_n}


def reduce_over_ranks(torch, dist, world, device, ms, work):
    """Weak scaling (one replica of the workload per rank): the slowest rank's time and the
    sum of every rank's work. Single process: the values themselves."""
    if world <= 1:
        return float(ms), float(work)
    tm = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tw = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(tw, op=dist.ReduceOp.SUM)
    return float(tm.item()), float(tw.item())


def run_ess(torch, L, S, step, stats, stream, n_sweeps, flags=0, pairs=None, group=None, units=None, keep=10,
            adapt=False, prefix=None):
    """ESS/s: integrated autocorrelation time of every cold walker's total log-likelihood
    (Eq. like on its residual) over n_sweeps sweeps (first quarter discarded). Optionally
    collects training pairs of the learned proposal after the burn-in and the cold slots' unit
    coordinates of the last `keep` sweeps (for the mixture refit) into `units` (outside the
    timing)."""
    nb = S["resid"].shape[2]
    nw = S["resid"].shape[0]
    lnl = torch.empty(nw, dtype=torch.float64, device=S["P"].device)
    rf = torch.empty((nw, 2, nb, 2), dtype=torch.float32, device=S["P"].device)
    series = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_sweeps = 0.0
    stats.zero_()
    for k in range(n_sweeps):
        e0.record(stream)
        if group is not None and k % group[2] == 0:   # (fraction, friends, sweeps between rebuilds)
            L.gbk_sweep_update_group(S["plan"], S["P"], S["E"], group[0], group[1], stream)
        step(flags)
        if adapt:   # every band's ladder from this sweep's swap acceptance (Vousden et al.)
            L.gbk_sweep_adapt_temps(S["plan"], S["betas"], k, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t_sweeps += e0.elapsed_time(e1) * 1e-3
        rf.copy_((S["resid"].to(torch.float64) * 2.0 ** -FRAC_BITS).to(torch.float32))
        L.total_loglike(S["ctx"], rf, S["psdp"].expand(nw, 2).contiguous(), lnl, stream)
        series.append(lnl.cpu().numpy().copy())
        if pairs is not None and k >= n_sweeps // 4 and pairs.n < pairs.capacity:
            pairs.add_from_sweep(S["plan"], S["P"], S["E"], S["R"], S["psd"])
        if units is not None and k >= n_sweeps - keep:
            d = S["plan"].desc
            u = torch.empty((d.n_walkers, d.n_bands, d.n_max, 8), dtype=torch.float32, device=S["P"].device)
            L.gb_sweep_features(S["plan"], S["P"], S["E"], S["R"], S["psd"], None, u, stream)
            units.append(u)
    st = stats.cpu().numpy()
    x = np.array(series).T[:, n_sweeps // 4:]
    tau = autocorr_time(x)
    n_eff = x.shape[0] * x.shape[1] / max(tau, 1.0)
    extra = {}
    if prefix is not None and prefix < n_sweeps:   # the same estimate from the first `prefix` sweeps only
        xp = np.array(series[:prefix]).T[:, prefix // 4:]
        tp = autocorr_time(xp)
        extra = {"prefix_sweeps": prefix, "tau_sweeps_prefix": tp,
                 "ess_per_s_prefix": xp.shape[0] * xp.shape[1] / max(tp, 1.0) / (t_sweeps / n_sweeps * xp.shape[1])}
    return {**extra, "ess_per_s": n_eff / (t_sweeps * x.shape[1] / n_sweeps), "tau_sweeps": tau, "sweeps": n_sweeps,
            "burn_in": n_sweeps // 4, "ms_per_sweep": 1e3 * t_sweeps / n_sweeps,
            "proposals_per_s": float(st[:4, 0].sum()) / t_sweeps,
            "acceptance": {k: float(st[i, 1]) / max(1.0, float(st[i, 0])) for i, k in
                           enumerate(["in_model", "birth", "death", "swap"])},
            "scalar": "cold-chain total lnL of each of the %d walkers (Eq. like on its residual)" % nw}


def recovered_sources(truth, P, E, tobs, n_bands, band_k0, walkers=4):
    """Injected sources matched by a cold-chain source of the same walker (|df0| < 1 bin,
    |d ln A| < 0.3), summed over the first `walkers` walkers."""
    f_t = truth[1] * tobs
    la_t = np.log(truth[0])
    bt = ((np.floor(f_t).astype(np.int64) - band_k0) // N_BAND)
    n = 0
    for w in range(min(walkers, P.shape[1])):
        for b in range(n_bands):
            sel = np.nonzero(bt == b)[0]
            if len(sel) == 0:
                continue
            cand = []
            for bb in (b - 1, b, b + 1):
                if 0 <= bb < n_bands:
                    m = E[0, w, bb].astype(bool)
                    cand.append(P[0, w, bb][m])
            c = np.concatenate(cand) if cand else np.zeros((0, 8))
            if len(c) == 0:
                continue
            df = np.abs(c[None, :, 1] * tobs - f_t[sel, None])
            da = np.abs(np.log(np.maximum(c[None, :, 0], 1e-30)) - la_t[sel, None])
            n += int(np.sum(np.any((df < 1.0) & (da < 0.3), axis=1)))
    return n


def run_gmm_fit(torch, L, units, n_walkers, args, stream):
    """Refit-RJ mixtures (Sec. V.E, App. G): one EM fit per band on the GPU to the cold-chain
    sources of the last sweeps, written as a sweep table [W][n_bands][272]; timed."""
    u = torch.stack(units)                                        # [keep][W][B][n_max][8]
    nb = u.shape[2]
    x = u.permute(2, 0, 1, 3, 4).reshape(nb, -1, 8).contiguous()  # [B][keep W n_max][8]
    raw = torch.empty((n_walkers, nb, 272), dtype=torch.float32, device=x.device)
    ll = torch.empty(nb, dtype=torch.float64, device=x.device)
    for _ in range(2):
        L.gmm_fit(x, raw, n_iter=args.gmm_iters, precision=L.GBK_MIXED, loglike=ll, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        L.gmm_fit(x, raw, n_iter=args.gmm_iters, precision=L.GBK_MIXED, loglike=ll, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    present = int((~torch.isnan(x).any(dim=2)).sum().item())
    used = int(torch.minimum((~torch.isnan(x).any(dim=2)).sum(dim=1),
                             torch.tensor(L.gmm_max_points(), device=x.device)).sum().item())
    return raw, {"bands": nb, "rows_per_band": int(x.shape[1]), "present_points": present, "fitted_points": used,
                 "components": 16, "em_iterations": args.gmm_iters, "sweeps_kept": len(units), "fit_ms": ms,
                 "point_iterations_per_s": used * (args.gmm_iters + 1) / (ms * 1e-3),
                 "precision": "mixed (float32 E-step, float64 M-step)"}


def run_search_rj(torch, L, S, ens, data, args, stream):
    """Search-RJ mixtures (Sec. V.E, App. G): every band's search sampler (4 temperatures x 32
    walkers, own-bin f0 prior) runs on walker 0's residual until its best point has not improved
    for n_it,max = 500 sweeps (App. G's convergence test; a converged band is left as it is),
    then every band relaunches from a ball around its best point and searches again until it
    converges; bands whose best point reaches SNR 7 give their cold walkers of 20 more sweeps to
    one EM fit per band; returns the sweep table [W][n_bands][272], the timings and the final
    walkers u [n_bands][4][32][8]."""
    dev = data.device
    nb, T_s, W_s = ens["n_bands"], 4, 32
    n_it_max = args.search_stall
    plan = L.SearchPlan(S["ctx"], nb, N_BAND, ens["band_k0"], T_s, W_s, L.GBK_MIXED, stall_limit=n_it_max)
    u = torch.empty((nb, T_s, W_s, 8), dtype=torch.float64, device=dev)
    ell = torch.empty((nb, T_s, W_s), dtype=torch.float64, device=dev)
    betas = torch.tensor([[0.5 ** t for t in range(T_s)]] * nb, dtype=torch.float64, device=dev)
    be = torch.full((nb,), -np.inf, dtype=torch.float64, device=dev)
    bu = torch.zeros((nb, 8), dtype=torch.float64, device=dev)
    stall = torch.zeros(nb, dtype=torch.int32, device=dev)
    st = torch.zeros((2, 2), dtype=torch.int64, device=dev)
    n_keep = 20
    x = torch.empty((nb, n_keep * W_s, 8), dtype=torch.float32, device=dev)
    key = 0x5EA2C4
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweep = [0]

    def until_converged(cap):
        # sweeps until every band has converged (checked every 50 sweeps) or `cap` sweeps
        n = 0
        while n < cap:
            for _ in range(50):
                L.gb_search_sweep(plan, u, ell, betas, S["psd"], key, sweep[0], best=(be, bu, stall), stats=st,
                                  stream=stream)
                sweep[0] += 1
                n += 1
            if int(stall.min().item()) >= n_it_max:
                break
        return n, int((stall >= n_it_max).sum().item())

    torch.cuda.synchronize()
    e0.record(stream)
    L.gb_search_init(plan, u, key, 1, stream)
    L.gb_search_windows(plan, L.residual_struct(data, FRAC_BITS), 0, stream)
    L.gb_search_eval(plan, u, ell, S["psd"], 0, stream)
    n1, conv1 = until_converged(args.search_rj_sweeps)
    snr1 = torch.sqrt(2.0 * torch.clamp(be, min=0.0)).cpu().numpy()
    # relaunch every band's ensemble from a ball around its best point (App. G), search again
    L.gb_search_ball(plan, u, be, bu, 0.002, key, 2, stream)
    L.gb_search_eval(plan, u, ell, S["psd"], 0, stream)
    stall.zero_()
    n2, conv2 = until_converged(args.search_rj_sweeps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_run = e0.elapsed_time(e1)
    stall.zero_()   # samples of every band (converged or not) for the mixtures
    for k in range(n_keep):
        L.gb_search_sweep(plan, u, ell, betas, S["psd"], key, sweep[0], best=(be, bu, stall), stream=stream)
        sweep[0] += 1
        L.gb_search_samples(plan, u, be, 7.0, F_LO, F_HI, x, k * W_s, stream)
    raw = torch.empty((N_W, nb, 272), dtype=torch.float32, device=dev)
    e0.record(stream)
    L.gmm_fit(x, raw, n_iter=args.gmm_iters, precision=L.GBK_MIXED, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    snr = torch.sqrt(2.0 * torch.clamp(be, min=0.0)).cpu().numpy()
    s = st.cpu().numpy()
    plan.close()
    out = {"bands": nb, "temps": T_s, "walkers": W_s, "n_it_max": n_it_max,
           "sweeps_to_convergence": n1, "bands_converged": conv1, "bands_snr_ge_7_before_relaunch": int((snr1 >= 7).sum()),
           "sweeps_after_relaunch": n2, "bands_converged_after_relaunch": conv2, "ball_sigma": 0.002,
           "sample_sweeps": n_keep, "ms_search": ms_run,
           "stretch_proposals_per_s": float(s[0, 0]) / (ms_run * 1e-3),
           "stretch_acceptance": float(s[0, 1]) / max(1.0, float(s[0, 0])),
           "swap_acceptance": float(s[1, 1]) / max(1.0, float(s[1, 0])),
           "bands_snr_ge_7": int((snr >= 7.0).sum()), "best_snr_median": float(np.median(snr)),
           "fit_ms": e0.elapsed_time(e1), "snr_min": 7.0}
    return raw, out, u


class WalkerSearch:
    """One search per walker, rerun as the fit proceeds (the paper keeps a search sampler per
    walker on that walker's current residual): a plan of N_W sets (4 temperatures x 32 walkers per
    band each). A rerun draws every set's walkers from the prior again, moves its windows to its
    walker's current residual and searches until every band has converged (n_it,max =
    args.search_rerun_stall sweeps without a better point, a converged band left as it is; at
    most args.search_rerun_sweeps sweeps), then fits the cold walkers of 20 more sweeps per
    (walker, band); returns the sweep table [N_W][n_bands][272]."""

    def __init__(self, torch, L, S, ens, args, stream):
        self.torch, self.L, self.S, self.args, self.stream = torch, L, S, args, stream
        dev = S["P"].device
        nb, self.T_s, self.W_s = ens["n_bands"], 4, 32
        self.nb = nb
        self.n_it = args.search_rerun_stall
        self.plan = L.SearchPlan(S["ctx"], nb, N_BAND, ens["band_k0"], self.T_s, self.W_s, L.GBK_MIXED,
                                 stall_limit=self.n_it, n_sets=N_W)
        self.u = torch.empty((N_W, nb, self.T_s, self.W_s, 8), dtype=torch.float64, device=dev)
        self.ell = torch.empty((N_W, nb, self.T_s, self.W_s), dtype=torch.float64, device=dev)
        self.betas = torch.tensor([[[0.5 ** t for t in range(self.T_s)]] * nb] * N_W, dtype=torch.float64, device=dev)
        self.be = torch.empty((N_W, nb), dtype=torch.float64, device=dev)
        self.bu = torch.zeros((N_W, nb, 8), dtype=torch.float64, device=dev)
        self.stall = torch.zeros((N_W, nb), dtype=torch.int32, device=dev)
        self.x = torch.empty((N_W * nb, 20 * self.W_s, 8), dtype=torch.float32, device=dev)
        self.raw = torch.empty((1, N_W * nb, 272), dtype=torch.float32, device=dev)
        self.sweep = 0
        self.ms, self.sweeps, self.snr7 = [], [], []

    def rerun(self, resid, n_keep=20):
        torch, L, st = self.torch, self.L, self.stream
        key = 0x5EA2C5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        L.gb_search_init(self.plan, self.u, key, 100 + len(self.ms), st)
        L.gb_search_windows(self.plan, L.residual_struct(resid, FRAC_BITS), 0, st)
        L.gb_search_eval(self.plan, self.u, self.ell, self.S["psd"], 0, st)
        self.be.fill_(-np.inf)
        self.stall.zero_()
        n = 0
        while n < self.args.search_rerun_sweeps:
            for _ in range(50):
                L.gb_search_sweep(self.plan, self.u, self.ell, self.betas, self.S["psd"], key, self.sweep,
                                  best=(self.be, self.bu, self.stall), stream=st)
                self.sweep += 1
                n += 1
            if int(self.stall.min().item()) >= self.n_it:
                break
        self.stall.zero_()   # samples of every band
        for k in range(n_keep):
            L.gb_search_sweep(self.plan, self.u, self.ell, self.betas, self.S["psd"], key, self.sweep,
                              best=(self.be, self.bu, self.stall), stream=st)
            self.sweep += 1
            L.gb_search_samples(self.plan, self.u, self.be, 7.0, F_LO, F_HI, self.x, k * self.W_s, st)
        L.gmm_fit(self.x, self.raw, n_iter=self.args.gmm_iters, precision=L.GBK_MIXED, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        self.ms.append(e0.elapsed_time(e1))
        self.sweeps.append(n)
        self.snr7.append(int((torch.sqrt(2.0 * torch.clamp(self.be, min=0.0)) >= 7.0).sum().item()))
        return self.raw.view(N_W, self.nb, 272)

    def close(self):
        self.plan.close()


def run_learned(torch, L, S, ens, step, stats, stream, sweep_no, args, pairs, snap, ess_plain, units=None):
    """The learned proposal on the ensemble: training throughput on the cold-chain pairs
    (BF16 tensor cores), then the same ESS run with the proposal, then a search from an
    empty model with and without it."""
    from paper_2405_04690_gb300 import proposal as PR
    dev = S["P"].device
    n = pairs.n
    n_val = max(4096, n // 20)
    n_tr = n - n_val
    batch = 4096
    train = PR.PairBuffer(1)
    train.x, train.u, train.n = pairs.x[:n_tr], pairs.u[:n_tr], n_tr
    val = PR.PairBuffer(1)
    val.x, val.u, val.n = pairs.x[n_tr:n], pairs.u[n_tr:n], n_val
    net = L.Mdn(max(batch, N_W * ((ens["n_bands"] + 1) // 2)))
    tr = PR.Trainer(net, torch.from_numpy(PR.init_params(11)).to(dev), lr=1e-3)
    v0 = tr.mean_loss(val)
    tr.epoch(train, batch, seed=0, max_steps=5)          # warm-up (also first steps of training)
    # the epochs' shuffled orders are drawn on the host before the timed region (a data loader's
    # work, ~20 ms per epoch of 950k pairs on the host, done ahead of the device like a prefetch)
    orders = [tr.order(train, batch, seed=1 + ep) for ep in range(args.mdn_epochs)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps0 = tr.step
    e0.record(stream)
    for o in orders:
        tr.epoch_ordered(train, o, batch)
    e1.record(stream)
    torch.cuda.synchronize()
    t_train = e0.elapsed_time(e1) * 1e-3
    samples = (tr.step - steps0) * batch
    v1 = tr.mean_loss(val)
    # inference throughput on batch-sized blocks
    raw = torch.empty((batch, PR.N_OUT), dtype=torch.float32, device=dev)
    for _ in range(3):
        L.mdn_forward(net, train.x[:batch], raw)
    e0.record(stream)
    reps = 50
    for r in range(reps):
        L.mdn_forward(net, train.x[(r % 8) * batch:(r % 8 + 1) * batch], raw)
    e1.record(stream)
    torch.cuda.synchronize()
    t_inf = e0.elapsed_time(e1) * 1e-3
    peak = None
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        peak = 1900.0
    tflops = samples * PR.FLOPS_TRAIN / t_train / 1e12
    out = {"pairs": n, "train_pairs": n_tr, "val_pairs": n_val, "batch": batch, "epochs": args.mdn_epochs,
           "train_samples_per_s": samples / t_train, "train_tflops": tflops,
           "train_roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                              "frac": tflops / peak, "peak_kind": "measured cuBLAS bf16 burst",
                              "flops_per_sample": PR.FLOPS_TRAIN},
           "infer_samples_per_s": reps * batch / t_inf,
           "infer_tflops": reps * batch * PR.FLOPS_FORWARD / t_inf / 1e12,
           "val_nll_start": v0, "val_nll_end": v1}
    # ESS with the learned proposal from the same starting state
    P0, E0, R0, k0 = snap
    S["P"].copy_(P0)
    S["E"].copy_(E0)
    S["resid"].copy_(R0)
    L.gbk_sweep_set_proposal(S["plan"], net=net, eps=args.mdn_eps, inmodel_frac=args.mdn_inmodel)
    sweep_no[0] = k0
    L.gb_sweep(S["plan"], S["P"], S["E"], S["betas"], S["R"], S["psd"], 1, 0, L.SWEEP_REFRESH, stream=stream)
    out["ess"] = run_ess(torch, L, S, step, stats, stream, args.ess_sweeps, flags=L.SWEEP_MDN)
    out["ess_gain"] = out["ess"]["ess_per_s"] / ess_plain["ess_per_s"]
    out["proposal"] = {"eps_prior": args.mdn_eps, "inmodel_frac": args.mdn_inmodel}
    # the paper's refit-RJ Gaussian mixtures as the comparison proposal: fitted on the GPU to
    # the last sweeps of the plain run, then the same ESS run with them
    gmm_raw = None
    if units:
        gmm_raw, gfit = run_gmm_fit(torch, L, units, N_W, args, stream)
        S["P"].copy_(P0)
        S["E"].copy_(E0)
        S["resid"].copy_(R0)
        L.gbk_sweep_set_proposal(S["plan"], raw_table=gmm_raw, eps=args.mdn_eps, inmodel_frac=args.mdn_inmodel)
        sweep_no[0] = k0
        L.gb_sweep(S["plan"], S["P"], S["E"], S["betas"], S["R"], S["psd"], 1, 0, L.SWEEP_REFRESH, stream=stream)
        gfit["ess"] = run_ess(torch, L, S, step, stats, stream, args.ess_sweeps, flags=L.SWEEP_MDN)
        gfit["ess_gain"] = gfit["ess"]["ess_per_s"] / ess_plain["ess_per_s"]
        out["gmm_refit"] = gfit
    # search: every chain starts empty (residual = data); K sweeps with each proposal
    search = {"sweeps": args.search_sweeps}
    L.gbk_sweep_set_proposal(S["plan"])
    S["P"].copy_(P0)
    S["E"].copy_(E0)
    S["resid"].copy_(R0)
    cold = P0[0].reshape(-1, 8)[E0[0].reshape(-1).bool()]
    wv = E0[0].reshape(N_W, -1).bool().nonzero()[:, 0].to(torch.int32)
    L.residual_add_sub(S["ctx"], S["R"], cold.t().contiguous(), torch.full((cold.shape[0],), N_BAND,
                       dtype=torch.int32, device=dev), N_BAND, wv, -1, L.GBK_MIXED, stream)
    data = S["resid"].clone()                               # d (noise + injected sources) per walker
    # the paper's search-RJ proposal: per-band search samplers on walker 0's data residual, then
    # mixtures fitted to their cold walkers around the best points of bands with SNR >= 7
    srj_raw, search["search_rj_sampler"], _ = run_search_rj(torch, L, S, ens, data, args, stream)
    walker_search = None
    for mode in ("prior", "learned", "gmm_refit", "search_rj", "search_rj_rerun"):
        if mode == "gmm_refit" and gmm_raw is None:
            continue
        S["P"].zero_()
        S["E"].zero_()
        S["resid"].copy_(data)
        if mode == "learned":
            L.gbk_sweep_set_proposal(S["plan"], net=net, eps=args.mdn_eps, inmodel_frac=args.mdn_inmodel)
        elif mode == "gmm_refit":
            L.gbk_sweep_set_proposal(S["plan"], raw_table=gmm_raw, eps=args.mdn_eps, inmodel_frac=args.mdn_inmodel)
        elif mode in ("search_rj", "search_rj_rerun"):
            L.gbk_sweep_set_proposal(S["plan"], raw_table=srj_raw, eps=args.mdn_eps, inmodel_frac=args.mdn_inmodel)
        else:
            L.gbk_sweep_set_proposal(S["plan"])
        fl = 0 if mode == "prior" else L.SWEEP_MDN
        stats.zero_()
        curve = []
        t = 0.0
        for k in range(args.search_sweeps):
            e0.record(stream)
            L.gb_sweep(S["plan"], S["P"], S["E"], S["betas"], S["R"], S["psd"], 0xA11, 5000 + k,
                       1 | 2 | 4 | fl | (L.SWEEP_REFRESH if k == 0 else 0), stats=stats, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) * 1e-3
            if k in (0, 1, 2, 4, args.search_sweeps - 1):
                curve.append([k + 1, recovered_sources(ens["truth"], S["P"].cpu().numpy(), S["E"].cpu().numpy(),
                                                       TOBS, ens["n_bands"], ens["band_k0"])])
            if mode == "search_rj_rerun" and k % 2 == 1 and k + 1 < args.search_sweeps:
                # the paper's continuous search: every walker's search continues on that walker's
                # current residual, so each band's search moves on to the loudest source not yet
                # in that walker's model, and each walker births from its own mixtures
                if walker_search is None:
                    walker_search = WalkerSearch(torch, L, S, ens, args, stream)
                srj_raw2 = walker_search.rerun(S["resid"])
                L.gbk_sweep_set_proposal(S["plan"], raw_table=srj_raw2, eps=args.mdn_eps,
                                         inmodel_frac=args.mdn_inmodel)
        st = stats.cpu().numpy()
        search[mode] = {"recovered_after_sweeps": curve, "seconds": t,
                        "birth_acceptance": float(st[1, 1]) / max(1.0, float(st[1, 0]))}
        if mode == "search_rj_rerun":
            search[mode]["reruns"] = ("after every second sweep, one search per walker (32 sets of 369 bands x 4 x 32) "
                                      "from the prior on that walker's current residual until converged "
                                      "(n_it,max %d, at most %d sweeps), then fitted (not in seconds)"
                                      % (args.search_rerun_stall, args.search_rerun_sweeps))
            if walker_search is not None:
                search[mode]["rerun_ms"] = walker_search.ms
                search[mode]["rerun_sweeps"] = walker_search.sweeps
                search[mode]["rerun_bands_snr_ge_7_all_walkers"] = walker_search.snr7
                walker_search.close()
    search["injected"] = int(ens["truth"].shape[1]) * min(4, N_W)
    search["counted"] = "cold chains of walkers 0-3: injected sources matched within 1 bin in f0 and 0.3 in ln A"
    out["search"] = search
    L.gbk_sweep_set_proposal(S["plan"])
    net.close()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()              # spawned pool, before any CUDA call
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_2405_04690_gb300 import _lib as L
    L.lib()
    ens = build_ensemble(seed=1 + 1000 * rank, n_temps=args.n_temps)
    S = build_device_state(torch, L, dev, ens, L.GBK_MIXED, seed=1 + 1000 * rank)
    stream = torch.cuda.current_stream()
    stats = torch.zeros((5, 2), dtype=torch.int64, device=dev)
    key = 0x5EED0000 + rank
    sweep_no = [0]

    xfer = torch.zeros(2, dtype=torch.int32, device=dev)   # ownership transfers: moved, blocked

    def step(flags_extra=0):
        # one sweep (in-model + flip-all RJ + swaps over both parities), then the band-edge
        # ownership transfer of the cold chain (Sec. V.D)
        L.gb_sweep(S["plan"], S["P"], S["E"], S["betas"], S["R"], S["psd"], key, sweep_no[0],
                   1 | 2 | 4 | flags_extra, stats=stats, stream=stream)
        L.gbk_sweep_transfer(S["plan"], S["P"], S["E"], xfer, stream)
        sweep_no[0] += 1

    step(L.SWEEP_REFRESH)                  # fills the waveform cache
    for _ in range(args.warmup):
        step()
    L.gbk_sync_status(S["ctx"])
    stats.zero_()
    xfer.zero_()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kms = np.zeros(4)
    clocks = ClockSampler()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for e0, e1 in evs:
        e0.record(stream)
        step(L.SWEEP_TIMING)
        e1.record(stream)
        kms += np.array(L.gbk_sweep_kernel_ms(S["plan"]))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    clk = clocks.stop(local)
    L.gbk_sync_status(S["ctx"])
    st = stats.cpu().numpy()
    xf = xfer.cpu().numpy()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    ms_step, total_props = reduce_over_ranks(torch, dist, world, dev, float(np.sum(ms)) / args.steps,
                                             float(st[:4, 0].sum()) / args.steps)
    value = total_props / (ms_step * 1e-3)
    # roofline of the band kernel (in-model + RJ): algorithmic flops / its device time
    wf, ev = float(st[4, 0]), float(st[4, 1])
    band_ms = kms[2] / args.steps
    # the short-series count where any source can take it: exact when every source does (this
    # ensemble: its band allowances end half a band above the last band, ~4.0 mHz, and the
    # chirp-mass prior's fdot adds < 1e-7 Hz over T), a lower bound otherwise
    f_top = (ens["band_k0"] + (ens["n_bands"] + 0.5) * N_BAND) / TOBS + 1e-7
    fl_wf = flops_per_waveform(N_BAND, short=short_series(F_LO))
    fl_note = "exact" if short_series(f_top) else "lower bound (sources on both sides of the short-series limit)"
    fl_step = (wf * fl_wf + ev * flops_per_evaluation()) / args.steps
    ach = fl_step / (band_ms * 1e-3) / 1e12

    # end to end through the C ABI with host buffers: the sampler state goes in from pinned
    # host memory and comes back (with the move statistics) every step
    Ph = S["P"].cpu().pin_memory()
    Eh = S["E"].cpu().pin_memory()
    sth = torch.zeros((5, 2), dtype=torch.int64).pin_memory()

    def e2e_step():
        S["P"].copy_(Ph, non_blocking=True)
        S["E"].copy_(Eh, non_blocking=True)
        step()
        Ph.copy_(S["P"], non_blocking=True)
        Eh.copy_(S["E"], non_blocking=True)
        sth.copy_(stats, non_blocking=True)

    torch.cuda.synchronize()
    stats.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms, e2e_props = reduce_over_ranks(torch, dist, world, dev, e0.elapsed_time(e1) / args.steps,
                                          float(stats[:4, 0].sum().item()) / args.steps)
    h2d = S["P"].numel() * 8 + S["E"].numel()
    d2h = h2d + 80

    # total log-likelihood pass of 512 walkers x 2 channels x 2^20 bins (float32 residual,
    # per-walker PSD; HBM bound): psd_eval for the noise draw, total_loglike timed
    c3 = {}
    if not args.no_c3:
        from paper_2405_04690_gb300 import synth
        g3 = synth.rng(3 + 1000 * rank)
        n3, w3, k03 = 1 << 20, args.c3_walkers, 3146
        ctx3 = L.Context(TOBS, DT, k03, n3)
        pp3 = torch.from_numpy(synth.draw_psd_params(g3, w3)).to(dev)
        r3 = torch.empty((w3, 2, n3, 2), dtype=torch.float32, device=dev)
        s3 = torch.empty((1, n3), dtype=torch.float64, device=dev)
        gen = torch.Generator(device=dev)
        gen.manual_seed(3 + 1000 * rank)
        for w in range(w3):
            L.psd_eval(ctx3, pp3[w:w + 1].contiguous(), s3)
            sd = torch.sqrt(s3[0] * (TOBS / 4.0)).to(torch.float32)
            r3[w].normal_(generator=gen)
            r3[w].mul_(sd[None, :, None])
        out3 = torch.empty(w3, dtype=torch.float64, device=dev)
        for _ in range(3):
            L.total_loglike(ctx3, r3, pp3, out3, stream)
        torch.cuda.synchronize()
        evs3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a0, a1 in evs3:
            a0.record(stream)
            L.total_loglike(ctx3, r3, pp3, out3, stream)
            a1.record(stream)
        torch.cuda.synchronize()
        ms3 = float(np.mean([a0.elapsed_time(a1) for a0, a1 in evs3]))
        bytes3 = w3 * 2 * n3 * 8
        peak, kind = measured_hbm_gbs()
        c3 = {"workload": "total logL: %d walkers x 2 ch x 2^20 bins float32, per-walker PSD (Eq. like)" % w3,
              "ms": ms3, "GB/s": bytes3 / (ms3 * 1e-3) / 1e9, "algorithmic_bytes": bytes3,
              "peak_GB/s": peak, "peak_kind": kind, "frac": bytes3 / (ms3 * 1e-3) / 1e9 / peak,
              "walker_logl_per_s": w3 / (ms3 * 1e-3)}
        # the PSD module (Sec. V.B): per-channel noise + Galactic foreground (9 parameters per
        # walker) over the same residuals; (a) one likelihood pass of all walkers, (b) sweeps of
        # the stretch/tempering sampler with 4 temperatures x 128 walkers (walker w's four
        # temperatures share residual w and read it once)
        g9 = synth.rng(9 + 1000 * rank)
        p9 = np.tile(np.array([15e-12, 3e-15, 15e-12, 3e-15, 3.3e-44, 1.2, 2.8e-3, 1763.3, 1686.3]), (w3, 1))
        p9[:, :4] *= np.exp(g9.uniform(-0.2, 0.2, (w3, 4)))
        pt9 = torch.from_numpy(p9).to(dev)
        out9 = torch.empty(w3, dtype=torch.float64, device=dev)
        for _ in range(3):
            L.total_loglike_fg(ctx3, r3, pt9, out9, stream=stream)
        torch.cuda.synchronize()
        for a0, a1 in evs3:
            a0.record(stream)
            L.total_loglike_fg(ctx3, r3, pt9, out9, stream=stream)
            a1.record(stream)
        torch.cuda.synchronize()
        ms9 = float(np.mean([a0.elapsed_time(a1) for a0, a1 in evs3]))
        c3["foreground"] = {"workload": "Eq. like with per-channel noise + Galactic foreground (9 parameters per "
                                        "walker), %d walkers x 2 ch x 2^20 bins" % w3,
                            "ms": ms9, "GB/s": bytes3 / (ms9 * 1e-3) / 1e9, "frac": bytes3 / (ms9 * 1e-3) / 1e9 / peak}
        T9, W9 = 4, min(128, w3)
        lo9 = np.array([math.log(5e-12), math.log(1e-15), math.log(5e-12), math.log(1e-15), math.log(1e-45), 0.8,
                        1e-3, 500.0, 500.0])
        hi9 = np.array([math.log(45e-12), math.log(9e-15), math.log(45e-12), math.log(9e-15), math.log(1e-42), 1.6,
                        4e-3, 3000.0, 3000.0])
        plan9 = L.PsdPlan(ctx3, T9, W9, lo9, hi9)
        ps9 = torch.from_numpy(np.stack([p9[:W9]] * T9)).to(dev).contiguous()
        ls9 = torch.empty((T9, W9), dtype=torch.float64, device=dev)
        rs9 = r3[:W9]
        L.total_loglike_fg(ctx3, rs9, ps9.reshape(T9 * W9, 9), ls9.reshape(-1),
                           resid_index=torch.arange(W9, dtype=torch.int32, device=dev).repeat(T9), stream=stream)
        bt9 = torch.from_numpy(np.array([1.2 ** -t for t in range(T9)])).to(dev)
        st9 = torch.zeros((2, 2), dtype=torch.int64, device=dev)
        for k in range(3):
            L.gb_psd_sweep(plan9, ps9, ls9, rs9, bt9, 0x9D, k, st9, stream)
        torch.cuda.synchronize()
        st9.zero_()
        n9 = 10
        a0, a1 = evs3[0]
        a0.record(stream)
        for k in range(n9):
            L.gb_psd_sweep(plan9, ps9, ls9, rs9, bt9, 0x9D, 3 + k, st9, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        ms_sw = a0.elapsed_time(a1) / n9
        s9 = st9.cpu().numpy()
        sweep_bytes = 2 * W9 // 2 * 2 * (1 << 20) * 8   # each half reads its W/2 residuals once
        c3["psd_sweep"] = {"workload": "PSD sampler sweep: %d temperatures x %d walkers, 2^20 bins, stretch moves of "
                                       "both halves + tempering swaps" % (T9, W9),
                           "ms_per_sweep": ms_sw, "walker_updates_per_s": T9 * W9 / (ms_sw * 1e-3),
                           "GB/s": sweep_bytes / (ms_sw * 1e-3) / 1e9,
                           "frac": sweep_bytes / (ms_sw * 1e-3) / 1e9 / peak,
                           # each half evaluates T x W/2 proposals over every bin; the four
                           # temperatures of a walker share its residual read, so the sweep is
                           # bound by the per-entry arithmetic (compare the foreground pass's rate)
                           "entry_bins_per_s": 2 * T9 * (W9 // 2) * (1 << 20) / (ms_sw * 1e-3),
                           "foreground_pass_entry_bins_per_s": w3 * (1 << 20) / (ms9 * 1e-3),
                           "stretch_acceptance": float(s9[0, 1]) / max(1.0, float(s9[0, 0])),
                           "swap_acceptance": float(s9[1, 1]) / max(1.0, float(s9[1, 0]))}
        plan9.close()
        del r3, s3
        ctx3.close()

    # uneven band lengths in one batch (200,000 proposals, f0 log-uniform in 0.3-20 mHz, N by
    # octave): binned by N, launch shape autotuned per N, the four launches captured in one
    # CUDA graph and replayed
    uneven = {}
    if not args.no_uneven:
        uneven = run_uneven(torch, L, dev, stream, seed=2 + 1000 * rank)

    # effective samples: integrated autocorrelation time of every cold walker's total
    # log-likelihood (Eq. like on its residual) over a run of sweeps
    ess = {}
    learned = {}
    if args.ess_sweeps > 0:
        snap = (S["P"].clone(), S["E"].clone(), S["resid"].clone(), sweep_no[0])
        pairs = None
        units = None
        if not args.no_learned:
            from paper_2405_04690_gb300 import proposal as PR
            pairs = PR.PairBuffer(args.mdn_samples)
            units = []
        ess = run_ess(torch, L, S, step, stats, stream, args.ess_sweeps, pairs=pairs, units=units,
                      keep=args.gmm_keep, prefix=args.fp64_sweeps)
        if args.group_frac > 0:   # the paper's in-model move: group stretch, group rebuilt every 30 sweeps
            S["P"].copy_(snap[0])
            S["E"].copy_(snap[1])
            S["resid"].copy_(snap[2])
            L.gb_sweep(S["plan"], S["P"], S["E"], S["betas"], S["R"], S["psd"], 1, 0, L.SWEEP_REFRESH, stream=stream)
            eg = run_ess(torch, L, S, step, stats, stream, args.ess_sweeps,
                         group=(args.group_frac, args.n_friends, 30))
            L.gbk_sweep_update_group(S["plan"], S["P"], S["E"], 0.0, 1, stream)
            eg["group"] = {"frac": args.group_frac, "n_friends": args.n_friends, "rebuild_every_sweeps": 30}
            eg["ess_gain"] = eg["ess_per_s"] / ess["ess_per_s"]
            ess["group_stretch"] = eg
        # ladders adapted after every sweep (the paper adapts its temperatures as it runs)
        betas0 = S["betas"].clone()
        S["P"].copy_(snap[0])
        S["E"].copy_(snap[1])
        S["resid"].copy_(snap[2])
        L.gb_sweep(S["plan"], S["P"], S["E"], S["betas"], S["R"], S["psd"], 1, 0, L.SWEEP_REFRESH, stream=stream)
        ea = run_ess(torch, L, S, step, stats, stream, args.ess_sweeps, adapt=True)
        bt = S["betas"].cpu().numpy()
        ea["ladder"] = {"beta_rung_1_median": float(np.median(bt[:, 1])), "beta_rung_1_range":
                        [float(bt[:, 1].min()), float(bt[:, 1].max())], "start_beta_rung_1": float(betas0[0, 1].item())}
        ea["ess_gain"] = ea["ess_per_s"] / ess["ess_per_s"]
        ess["adaptive_ladder"] = ea
        S["betas"].copy_(betas0)
        if pairs is not None:
            learned = run_learned(torch, L, S, ens, step, stats, stream, sweep_no, args, pairs, snap, ess, units)
        del snap

    # the paper's schedule (Sec. V.D): ~30 in-model proposals per source, then the RJ pass and
    # the swaps, on the same ensemble (own plan, refreshed from the current state)
    sched30 = {}
    if args.pps30_sweeps > 0:
        plan30 = L.SweepPlan(S["ctx"], ens["params"].shape[0], N_W, ens["n_bands"], ens["n_max"], N_BAND,
                             ens["band_k0"], sweep_sigma(), L.GBK_MIXED, f_min=F_LO, f_max=F_HI, props_per_source=30.0)
        S30 = dict(S)
        S30["plan"] = plan30
        sw30 = [sweep_no[0]]

        def step30(flags_extra=0):
            L.gb_sweep(plan30, S30["P"], S30["E"], S30["betas"], S30["R"], S30["psd"], key, sw30[0],
                       1 | 2 | 4 | flags_extra, stats=stats, stream=stream)
            L.gbk_sweep_transfer(plan30, S30["P"], S30["E"], xfer, stream)
            sw30[0] += 1

        step30(L.SWEEP_REFRESH)
        step30()
        torch.cuda.synchronize()
        sched30 = run_ess(torch, L, S30, step30, stats, stream, args.pps30_sweeps)
        st30 = stats.cpu().numpy()
        sched30["waveforms_per_s"] = float(st30[4, 0]) / (sched30["ms_per_sweep"] * 1e-3 * args.pps30_sweeps)
        sched30["schedule"] = "30 in-model proposals per source, then flip-all RJ, then tempering swaps (Sec. V.D)"
        plan30.close()

    # the plain float64 path on the same GPU: (a) the same sweep in float64, with its ESS/s
    # measured over a run of sweeps; (b) one float64 Delta lnL launch per source band carrying
    # that band's in-model proposals (every source moved, new != old), no batching across bands
    fp64 = {}
    if not args.no_fp64:
        S64 = build_device_state(torch, L, dev, ens, L.GBK_FP64, seed=1 + 1000 * rank)
        st64 = torch.zeros((5, 2), dtype=torch.int64, device=dev)
        sw64 = [0]

        def step64(flags_extra=0):
            L.gb_sweep(S64["plan"], S64["P"], S64["E"], S64["betas"], S64["R"], S64["psd"], key, sw64[0],
                       1 | 2 | 4 | flags_extra, stats=st64, stream=stream)
            L.gbk_sweep_transfer(S64["plan"], S64["P"], S64["E"], xfer, stream)
            sw64[0] += 1

        step64(L.SWEEP_REFRESH)
        torch.cuda.synchronize()
        e64 = run_ess(torch, L, S64, step64, st64, stream, args.fp64_sweeps)
        s64 = st64.cpu().numpy()
        fp64["fp64_sweep_proposals_per_s"] = e64["proposals_per_s"]
        fp64["fp64_sweep"] = {"ess_per_s": e64["ess_per_s"], "tau_sweeps": e64["tau_sweeps"],
                              "sweeps": e64["sweeps"], "ms_per_sweep": e64["ms_per_sweep"],
                              "proposals_per_s": e64["proposals_per_s"],
                              "waveforms_per_s": float(s64[4, 0]) / (e64["ms_per_sweep"] * 1e-3 * e64["sweeps"])}
        # per-band launches on walker 0's cold chain: bands in order, each band's present sources
        # moved by the sweep's in-model widths (Gaussian steps; ln A, f0, fdot, angles)
        g64 = np.random.default_rng(64 + 1000 * rank)
        sig = np.asarray(sweep_sigma())
        P0 = S64["P"][0, 0].cpu().numpy()
        E0 = S64["E"][0, 0].cpu().numpy().astype(bool)
        launches = []
        for b in range(ens["n_bands"]):
            old = P0[b][E0[b]]
            if len(old) == 0:
                continue
            new = old.copy()
            new[:, 0] = old[:, 0] * np.exp(sig[0] * g64.standard_normal(len(old)))
            new[:, 1:] = old[:, 1:] + sig[1:] * g64.standard_normal((len(old), 7))
            new[:, 3] %= 2 * math.pi
            new[:, 4] %= math.pi
            new[:, 7] %= 2 * math.pi
            new[:, 5:7] = np.clip(new[:, 5:7], -1.0, 1.0)
            launches.append((torch.from_numpy(np.ascontiguousarray(new.T)).to(dev),
                             torch.from_numpy(np.ascontiguousarray(old.T)).to(dev),
                             torch.full((len(old),), N_BAND, dtype=torch.int32, device=dev),
                             torch.zeros(len(old), dtype=torch.int32, device=dev),
                             torch.empty(len(old), dtype=torch.float64, device=dev)))
        for pn, po, nbv, wv, ov in launches[:5]:
            L.gb_delta_loglike_batch(S64["ctx"], pn, po, nbv, N_BAND, wv, S64["R"], S64["psd"], ov, L.GBK_FP64, stream)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for pn, po, nbv, wv, ov in launches:
            L.gb_delta_loglike_batch(S64["ctx"], pn, po, nbv, N_BAND, wv, S64["R"], S64["psd"], ov, L.GBK_FP64, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        n_prop = sum(int(x[4].numel()) for x in launches)
        fp64["fp64_per_band_proposals_per_s"] = n_prop / (a0.elapsed_time(a1) * 1e-3)
        fp64["fp64_per_band"] = {"launches": len(launches), "proposals": n_prop,
                                 "ms": a0.elapsed_time(a1),
                                 "path": "gb_delta_loglike_batch in float64, one launch per source band (walker 0, "
                                         "cold chain), each present source moved (new != old); two waveforms and "
                                         "one Delta lnL per proposal"}
        S64["plan"].close()
        del S64
    line = {
        "metric": METRIC, "value": value, "unit": "proposals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic: seeded noise + injected GBs drawn from the configured priors (LDC2A data not available)",
        "config": {"workload": WORKLOAD, "n_temps": int(args.n_temps), "n_walkers": N_W, "gbs_per_walker": N_SRC,
                   "band_bins": N_BAND, "n_bands": ens["n_bands"], "slots_per_band": ens["n_max"],
                   "precision": "mixed", "l2": "working set > L2 (16 GB waveform cache, 0.25 GB params); no flush",
                   "proposals_per_step": {"in_model": float(st[0, 0]) / args.steps,
                                          "birth": float(st[1, 0]) / args.steps,
                                          "death": float(st[2, 0]) / args.steps,
                                          "swap": float(st[3, 0]) / args.steps},
                   "acceptance": {k: (float(st[i, 1]) / max(1.0, float(st[i, 0]))) for i, k in
                                  enumerate(["in_model", "birth", "death", "swap"])},
                   "waveforms_per_step": wf / args.steps,
                   "ownership_transfers_per_step": {"moved": float(xf[0]) / args.steps,
                                                    "blocked": float(xf[1]) / args.steps},
                   "kernel_ms_per_step": {"open": kms[1] / args.steps, "band": band_ms, "swap": kms[3] / args.steps},
                   "parallelism": "replica per GPU"},
        "roofline": {"bound": "alu", "achieved": ach, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach / PEAK_FP32_TFLOPS, "traffic": K_BAND_TRAFFIC,
                     "traffic_note": "bytes per launch: ncu dram read + write of one k_band launch on the "
                                     "2-temperature ensemble (1.918 GB) x 8 for the 16-temperature launch "
                                     "(traffic scales with the band tasks)",
                     "kernel": "k_band<float,256> (in-model + flip-all RJ)",
                     "peak_note": "FP32 ALU: 152 SMs x 128 lanes x 2 (FMA) x 2.07 GHz (derived, not measured)",
                     "flops_per_waveform": fl_wf, "flops_per_evaluation": flops_per_evaluation(),
                     "flops_count": fl_note},
        "waveforms_per_s": wf / args.steps / (ms_step * 1e-3),
        "e2e": {"value": e2e_props / (e2e_ms * 1e-3), "unit": "proposals/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 9 * args.steps,   # per step: open, band, swap per parity; transfer assign, apply, sums
        "clocks": clk,
        "wall_s_timed_region": wall,
    }
    line["config"].update(fp64)
    if fp64:
        # ESS/s ratio on equal footing: the mixed sweep's estimate from its first fp64_sweeps sweeps
        # (same estimator, same run length as the float64 run)
        line["vs_plain_fp64"] = {
            "batched_mixed_over_fp64_sweep_proposals": value / fp64["fp64_sweep_proposals_per_s"],
            "batched_mixed_over_fp64_per_band_proposals": value / fp64["fp64_per_band_proposals_per_s"],
            "ess_per_s_mixed_over_fp64_sweep_same_run_length":
                (ess["ess_per_s_prefix"] / fp64["fp64_sweep"]["ess_per_s"]) if ess and "ess_per_s_prefix" in ess else None}
    if sched30:
        line["schedule_30_1_1"] = sched30
    if c3:
        line["total_loglike"] = c3
    if uneven:
        line["uneven_n"] = uneven
    if ess:
        line["ess"] = ess
    if learned:
        line["learned_proposal"] = learned
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    S["plan"].close()
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(n_bands=2)
    vals, walls = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        vals.append(cpu_baseline(n_bands=4))
        walls.append(time.perf_counter() - t0)
    v = float(np.mean([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    # n_gpus is the launch's N; the oracle itself runs on the host cores only (gpus_used 0), and
    # ms_per_step is the wall time of one bounded sample step (pool start included)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "proposals/s", "n_gpus": args.gpus,
            "gpus_used": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(walls)) if walls else None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (each step a bounded sample: one oracle sweep of 4 sub-bands per "
                                              "host core)"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "proposals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_kernel_case(args):
    """One small workload of a single kernel, for profiler captures (no JSON line):
    total_loglike: three total_loglike calls on 64 walkers x 2 ch x 2^20 bins (1.07 GB of float32
    residual, larger than L2); dlogl_1024: three Delta lnL batches of 20,000 proposals with
    1024-bin bands (f0 log-uniform in 4-20 mHz, one walker's zero residual), mixed precision;
    total_loglike_fg: three total_loglike_fg calls (per-channel noise + Galactic foreground, 9
    parameters per walker) on the same 64-walker residual size;
    mdn_train: the learned proposal's network on 40,960 random pairs, batch 4096: device times
    of the forward pass, forward + backward, the Adam step and one step of a training epoch
    (printed as one JSON line, microseconds)."""
    import torch
    from paper_2405_04690_gb300 import _lib as L
    from paper_2405_04690_gb300 import synth
    dev = torch.device("cuda")
    if args.kernel_case == "total_loglike":
        g = synth.rng(3)
        n, w, k0 = 1 << 20, 64, 3146
        ctx = L.Context(TOBS, DT, k0, n)
        pp = torch.from_numpy(synth.draw_psd_params(g, w)).to(dev)
        gen = torch.Generator(device=dev)
        gen.manual_seed(3)
        r = torch.randn((w, 2, n, 2), dtype=torch.float32, device=dev, generator=gen) * 1e-17
        out = torch.empty(w, dtype=torch.float64, device=dev)
        for _ in range(3):
            L.total_loglike(ctx, r, pp, out)
    elif args.kernel_case == "total_loglike_fg":
        g = synth.rng(9)
        n, w, k0 = 1 << 20, 64, 3146
        ctx = L.Context(TOBS, DT, k0, n)
        p9 = np.tile(np.array([15e-12, 3e-15, 15e-12, 3e-15, 3.3e-44, 1.2, 2.8e-3, 1763.3, 1686.3]), (w, 1))
        p9[:, :4] *= np.exp(g.uniform(-0.2, 0.2, (w, 4)))
        gen = torch.Generator(device=dev)
        gen.manual_seed(9)
        r = torch.randn((w, 2, n, 2), dtype=torch.float32, device=dev, generator=gen) * 1e-17
        out = torch.empty(w, dtype=torch.float64, device=dev)
        for _ in range(3):
            L.total_loglike_fg(ctx, r, torch.from_numpy(p9).to(dev), out)
    elif args.kernel_case == "mdn_train":
        from paper_2405_04690_gb300 import proposal as PR
        batch, n = 4096, 40960
        gen = torch.Generator(device=dev)
        gen.manual_seed(7)
        buf = PR.PairBuffer(n)
        buf.x.copy_(torch.randn((n, PR.N_IN), device=dev, generator=gen).to(torch.bfloat16))
        buf.u.copy_(torch.rand((n, PR.N_DIM), device=dev, generator=gen) * 0.98 + 0.01)
        buf.n = n
        net = L.Mdn(batch)
        tr = PR.Trainer(net, torch.from_numpy(PR.init_params(11)).to(dev), lr=1e-3)
        tr.epoch(buf, batch, seed=0, max_steps=3)
        raw = torch.empty((batch, PR.N_OUT), dtype=torch.float32, device=dev)
        grad = torch.empty_like(tr.p)
        x, u = buf.x[:batch], buf.u[:batch]
        st = torch.cuda.current_stream()
        times = {}
        for name, fn in (("forward", lambda: L.mdn_forward(net, x, raw)),
                         ("forward_backward", lambda: L.mdn_backward(net, x, u, grad)),
                         ("adam", lambda: L.mdn_adam(net, tr.p, tr.m, tr.v, grad, 10, 1e-3)),
                         ("train_epoch_step", lambda: tr.epoch(buf, batch, seed=1))):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 1 if name == "train_epoch_step" else 20
            e0.record(st)
            for _ in range(reps):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
            per = e0.elapsed_time(e1) * 1e3 / reps
            times[name] = per / (n // batch) if name == "train_epoch_step" else per
        # host time to enqueue one epoch (the call returns before the device finishes)
        order = torch.arange(n, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.mdn_train_epoch(net, tr.p, tr.m, tr.v, buf.x, buf.u, order, batch, 100, 1e-3)
        t1 = time.perf_counter()
        torch.cuda.synchronize()
        times["host_enqueue_per_step"] = (t1 - t0) * 1e6 / (n // batch)
        print(json.dumps({"mdn_train_us": times, "batch": batch}))
    else:
        g = synth.rng(5)
        m = 20000
        p = synth.draw_sources(g, m, 4e-3, 2e-2, log_f=True)
        new = synth.perturb(g, p, synth.proposal_widths(p))
        k0, nbins = synth.window_for(3.9e-3, 2.05e-2, 1100)
        ctx = L.Context(TOBS, DT, k0, nbins)
        psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
        resid = torch.zeros((1, 2, nbins, 2), dtype=torch.int64, device=dev)
        pn = torch.from_numpy(np.ascontiguousarray(new)).to(dev)
        po = torch.from_numpy(np.ascontiguousarray(p)).to(dev)
        nb = torch.full((m,), 1024, dtype=torch.int32, device=dev)
        wk = torch.zeros(m, dtype=torch.int32, device=dev)
        out = torch.empty(m, dtype=torch.float64, device=dev)
        for _ in range(3):
            L.gb_delta_loglike_batch(ctx, pn, po, nb, 1024, wk, L.residual_struct(resid, FRAC_BITS), L.psd_struct(psdp),
                                     out, L.GBK_MIXED)
    torch.cuda.synchronize()
    if args.kernel_case == "mdn_train":
        L.mdn_status(net)
    else:
        L.gbk_sync_status(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel-case", choices=["total_loglike", "total_loglike_fg", "dlogl_1024", "mdn_train"],
                    default=None,
                    help="run one small single-kernel workload for a profiler capture and exit")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64 comparison runs")
    ap.add_argument("--fp64-sweeps", type=int, default=48, help="sweeps of the float64 ESS run")
    ap.add_argument("--pps30-sweeps", type=int, default=40,
                    help="sweeps of the 30-in-model-proposals-per-source schedule (0: skip)")
    ap.add_argument("--no-c3", action="store_true", help="skip the total log-likelihood (HBM) measurement")
    ap.add_argument("--ess-sweeps", type=int, default=120, help="sweeps for the ESS/s measurement (0: skip)")
    ap.add_argument("--c3-walkers", type=int, default=512, help="walkers of the total log-likelihood measurement")
    ap.add_argument("--no-uneven", action="store_true", help="skip the uneven band-length measurement")
    ap.add_argument("--n-temps", type=int, default=N_T, help="smaller ensemble for profiling captures")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal measurements")
    ap.add_argument("--mdn-samples", type=int, default=1000000, help="training pairs of the learned proposal")
    ap.add_argument("--mdn-epochs", type=int, default=6)
    ap.add_argument("--mdn-eps", type=float, default=0.2, help="prior fraction of the learned proposal")
    ap.add_argument("--mdn-inmodel", type=float, default=0.1, help="fraction of in-model moves drawn from it")
    ap.add_argument("--search-sweeps", type=int, default=10)
    ap.add_argument("--gmm-keep", type=int, default=10, help="sweeps of cold-chain sources for the mixture refit")
    ap.add_argument("--search-rj-sweeps", type=int, default=3000,
                    help="cap on the search-sampler sweeps of each phase (before and after the relaunch)")
    ap.add_argument("--search-stall", type=int, default=500, help="n_it,max of the search's convergence test")
    ap.add_argument("--search-rerun-stall", type=int, default=100,
                    help="n_it,max of the per-walker search reruns during the search from an empty model")
    ap.add_argument("--search-rerun-sweeps", type=int, default=600, help="sweep cap of each per-walker search rerun")
    ap.add_argument("--gmm-iters", type=int, default=50, help="EM iterations of the mixture refit")
    ap.add_argument("--group-frac", type=float, default=0.5, help="fraction of in-model moves that are group stretches "
                                                                   "in the group-stretch ESS run (0: skip it)")
    ap.add_argument("--n-friends", type=int, default=32)
    args = ap.parse_args()
    if args.kernel_case:
        run_kernel_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
