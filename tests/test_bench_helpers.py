"""The benchmark's own statistics on the CPU: the integrated autocorrelation time behind the
ESS/s figures is checked on AR(1) chains, whose time is known in closed form,
tau = (1 + phi) / (1 - phi)."""
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
