"""Benchmark of the GB likelihood hot path on GB300 (one JSON line on stdout).

Workload: the batched ensemble of 16 temperatures x 32 walkers, each walker holding
2,000 Galactic binaries in 1-4 mHz with N = 256 band bins (1,024,000 sources), data =
seeded noise + 2,000 injected sources, residual of every walker on the device as int64
fixed point. One step evaluates one in-model Gaussian proposal for every source (S1-S5:
slow-part response, band FFT, heterodyne, PSD weights, Delta lnL against the walker's
residual) in mixed precision in one launch.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own replica of the workload (weak scaling); rank 0
prints max-over-ranks timing.
"""
import argparse
import json
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
METRIC = "GB proposals (waveform+DeltalogL) /sec"
WORKLOAD = "16 temps x 32 walkers x 2000 GBs (1-4 mHz, N=256): one in-model proposal per source, mixed precision"

# Algorithmic FP32 work of one in-model proposal at N = 256 (two waveforms and the
# inner products over the union of the two bands), counted from the algorithm:
# slow part 417 flops/sample, FFT 5 N log2 N per channel, 45 flops per union bin.
FLOPS_SLOW_PER_SAMPLE = 417
FLOPS_PER_BIN = 45


def flops_per_proposal(n=N_BAND, union_bins=N_BAND + 4):
    wf = n * FLOPS_SLOW_PER_SAMPLE + 2 * 5 * n * int(np.log2(n))
    return 2 * wf + union_bins * FLOPS_PER_BIN


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ CPU oracle timing
def _oracle_worker(args):
    seed, count = args
    sys.path.insert(0, ROOT)
    from oracle import constants as OC
    from oracle import likelihood as OL
    from oracle import psd as OP
    from oracle import waveform as OW
    from paper_2405_04690_gb300 import synth
    g = synth.rng(seed)
    p = synth.draw_sources(g, count)
    new = synth.perturb(g, p, synth.proposal_widths(p))
    t0 = time.perf_counter()
    for i in range(count):
        q, _ = OW.carrier_bin(p[1, i])
        k0 = q - 3 * N_BAND // 2
        f = (k0 + np.arange(3 * N_BAND)) * OC.DF
        s = OP.psd_ae(f, OC.SQRT_S_OMS, OC.SQRT_S_ACC)
        r = synth.unit_complex_normal(g, (2, 3 * N_BAND)) * np.sqrt(s / (4 * OC.DF))
        OL.delta_loglike_swap(r, s, OC.DF, k0, OW.fastslow_band(new[:, i], N_BAND), OW.fastslow_band(p[:, i], N_BAND))
    return time.perf_counter() - t0, count


def cpu_baseline(sample=4000, cores=None):
    """Time the FP64 oracle on `sample` proposals spread over all host cores (spawned pool)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    per = [sample // cores + (1 if i < sample % cores else 0) for i in range(cores)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(7000 + i, c) for i, c in enumerate(per) if c > 0])
    wall = time.perf_counter() - t0
    done = sum(c for _, c in res)
    busy = max(t for t, _ in res)
    return {"value": done / busy, "unit": "proposals/s", "cores": cores, "kind": "oracle",
            "sample": "%d in-model proposals (N=256, 1-4 mHz) over %d processes; FP64 numpy fast/slow waveform x2 + "
                      "Eq. swapsource on a 3-band window; %.1f s wall incl. pool start" % (done, cores, wall)}


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
def build_workload(torch, L, dev, seed, n_temps=N_T):
    from paper_2405_04690_gb300 import synth
    g = synth.rng(seed)
    k0, nbins = synth.window_for(1e-3, 4e-3, 600)
    ctx = L.Context(TOBS, DT, k0, nbins)
    truth = synth.draw_sources(g, N_SRC)
    psdp = torch.tensor([[synth.SQRT_S_OMS, synth.SQRT_S_ACC]], dtype=torch.float64, device=dev)
    # noise on the window: unit normals scaled by sqrt(S / 4df), S from psd_eval
    s = torch.empty((1, nbins), dtype=torch.float64, device=dev)
    L.psd_eval(ctx, psdp, s)
    z = torch.from_numpy(synth.unit_complex_normal(g, (2, nbins))).to(dev)
    noise = z * torch.sqrt(s[0] * (TOBS / 4.0))
    scale = float(2.0 ** FRAC_BITS)
    one = torch.stack([torch.round(noise.real * scale), torch.round(noise.imag * scale)], dim=-1).to(torch.int64)
    resid = one.unsqueeze(0).repeat(N_W, 1, 1, 1).contiguous()            # [W][2][n][2]
    R = L.residual_struct(resid, FRAC_BITS)
    nb = torch.full((N_SRC,), N_BAND, dtype=torch.int32, device=dev)
    # data = noise + injected truth (templates leave the model: R += h)
    for w in range(N_W):
        L.residual_add_sub(ctx, R, torch.from_numpy(truth).to(dev), nb, N_BAND,
                           torch.full((N_SRC,), w, dtype=torch.int32, device=dev), -1, L.GBK_MIXED)
    # per (t, w): walker-specific small jitter of the truth; cold chain (t = 0) is the model
    widths = synth.proposal_widths(truth) * 0.2
    cur = np.empty((8, n_temps * N_W * N_SRC))
    walker = np.empty(n_temps * N_W * N_SRC, dtype=np.int32)
    for t in range(n_temps):
        for w in range(N_W):
            i0 = (t * N_W + w) * N_SRC
            cur[:, i0:i0 + N_SRC] = synth.perturb(g, truth, widths)
            walker[i0:i0 + N_SRC] = w
    for w in range(N_W):
        i0 = w * N_SRC
        L.residual_add_sub(ctx, R, torch.from_numpy(np.ascontiguousarray(cur[:, i0:i0 + N_SRC])).to(dev), nb, N_BAND,
                           torch.full((N_SRC,), w, dtype=torch.int32, device=dev), +1, L.GBK_MIXED)
    L.gbk_sync_status(ctx)
    prop = synth.perturb(g, cur, synth.proposal_widths(cur))
    n = cur.shape[1]
    w_ = {
        "ctx": ctx, "resid": resid, "R": R, "psd": L.psd_struct(psdp), "psdp": psdp,
        "old": torch.from_numpy(cur).to(dev), "new": torch.from_numpy(prop).to(dev),
        "old_h": torch.from_numpy(cur).pin_memory(), "new_h": torch.from_numpy(prop).pin_memory(),
        "nb": torch.full((n,), N_BAND, dtype=torch.int32, device=dev),
        "walker": torch.from_numpy(walker).to(dev), "out": torch.empty(n, dtype=torch.float64, device=dev),
        "out_h": torch.empty(n, dtype=torch.float64).pin_memory(), "n": n,
    }
    return w_


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
    W = build_workload(torch, L, dev, seed=1 + 1000 * rank, n_temps=args.n_temps)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def step():
        L.gb_delta_loglike_batch(W["ctx"], W["new"], W["old"], W["nb"], N_BAND, W["walker"], W["R"], W["psd"],
                                 W["out"], L.GBK_MIXED, stream)

    for _ in range(args.warmup):
        step()
    L.gbk_sync_status(W["ctx"])
    launches = 0
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for e0, e1 in evs:
        flush.fill_(1.0)                    # untimed L2 flush between timed steps
        e0.record(stream)
        step()
        launches += 1
        e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    clk = clocks.stop(local)
    L.gbk_sync_status(W["ctx"])
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    ms_step = float(np.sum(ms)) / args.steps
    t = torch.tensor([ms_step], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_step = float(t.item())
    total_props = W["n"] * world
    value = total_props / (ms_step * 1e-3)

    # end to end through the C ABI with host buffers (H2D params, D2H Delta lnL)
    def e2e_step():
        W["new"].copy_(W["new_h"], non_blocking=True)
        W["old"].copy_(W["old_h"], non_blocking=True)
        step()
        W["out_h"].copy_(W["out"], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e_ms_t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_ms_t, op=dist.ReduceOp.MAX)
    e2e_ms = float(e2e_ms_t.item())
    fl = flops_per_proposal()
    peak_alu = 152 * 128 * 2 * 2.07e9 / 1e12     # FP32 lanes x FMA x max SM clock
    ach = fl * W["n"] / (float(np.mean(ms)) * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "proposals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded noise + injected GBs; LDC2A not available)",
        "config": {"workload": WORKLOAD, "global_batch": total_props, "n_temps": N_T, "n_walkers": N_W,
                   "n_sources_per_walker": N_SRC, "band_bins": N_BAND, "precision": "mixed",
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replica per GPU"},
        "roofline": {"bound": "alu", "achieved": ach, "peak": peak_alu, "unit": "TFLOP/s", "frac": ach / peak_alu,
                     "traffic": None,
                     "peak_note": "FP32: 152 SMs x 128 lanes x 2 (FMA) x 2.07 GHz; kernel k_dlogl<float,256>",
                     "flops_per_proposal": fl},
        "e2e": {"value": total_props / (e2e_ms * 1e-3), "unit": "proposals/s",
                "h2d_bytes_per_step": 2 * 8 * 8 * W["n"], "d2h_bytes_per_step": 8 * W["n"]},
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed_region": wall,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per = []
    for _ in range(args.warmup):
        cpu_baseline(sample=400)
    vals = [cpu_baseline(sample=800) for _ in range(args.steps)]
    v = float(np.mean([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "proposals/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (each step a bounded sample of 800 proposals on the host cores)"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "proposals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-temps", type=int, default=N_T, help="smaller ensemble for profiling captures")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
