"""The benchmark's own statistics on the CPU: the integrated autocorrelation time behind the
ESS/s figures is checked on AR(1) chains, whose time is known in closed form,
tau = (1 + phi) / (1 - phi); the clock sampler's parsing of nvidia-smi rows; the reference arm
(the oracle on the host cores) prints its one line on rank 0 only."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_autocorrelation_time_of_ar1_chains():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as BN
    g = np.random.default_rng(6)
    for phi in (0.0, 0.5, 0.8, 0.9):
        n_chains, n = 32, 20000
        x = np.empty((n_chains, n))
        x[:, 0] = g.standard_normal(n_chains) / np.sqrt(1 - phi ** 2)
        e = g.standard_normal((n_chains, n))
        for i in range(1, n):
            x[:, i] = phi * x[:, i - 1] + e[:, i]
        want = (1 + phi) / (1 - phi)
        got = BN.autocorr_time(x)
        assert abs(got / want - 1) < 0.1, (phi, got, want)


def test_clock_sampler_reads_median_and_throttle_reasons(tmp_path):
    # nvidia-smi CSV rows (index, sm, max sm, power, active mask, hw, hw thermal, sw thermal,
    # sw power cap): the median SM clock of GPU 0 and every reason seen active
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as BN

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    p = tmp_path / "clocks.csv"
    p.write_text("0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "1, 1000, 2070, 500, 0x0, Active, Not Active, Not Active, Not Active\n"
                 "0, 1980, 2070, 1400, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 2070, 2070, 1300, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    cs = BN.ClockSampler()
    cs.proc, cs.path = _Proc(), str(p)
    out = cs.stop(0)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_reference_arm_prints_one_line_on_rank_0_only():
    # the oracle timed on the host cores: one JSON line with the contract's keys on rank 0; any
    # other rank exits 0 without work or output
    import json
    import subprocess
    env = dict(os.environ, RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--gpus", "2"], capture_output=True, text=True, env=env, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["gpus_used"] == 0 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    env["RANK"] = "1"
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0 and out.stdout.strip() == ""
