"""Shared setup of the tests: seeded workloads built with the oracle and the synth module."""
import numpy as np
import pytest

from oracle import constants as OC
from oracle import psd as OP
from oracle import residual as OR
from paper_2405_04690_gb300 import synth

FRAC_BITS = 98            # residual grid 2^-98: the noise RMS near 2.5 mHz is ~2^40 units


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2405_04690_gb300 import _lib
    _lib.lib()  # fails loudly if the library is not built
    return torch


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def window(f_lo=1e-3, f_hi=4e-3, margin=600):
    return synth.window_for(f_lo, f_hi, margin)


def psd_window(k0, n, sqrt_oms=OC.SQRT_S_OMS, sqrt_acc=OC.SQRT_S_ACC):
    f = (k0 + np.arange(n)) * OC.DF
    return OP.psd_ae(f, sqrt_oms, sqrt_acc)


def noise_fixed(g, k0, n, s, frac=FRAC_BITS):
    """Seeded noise realisation of PSD s on the window, as int64 fixed point [2][n][2]."""
    z = synth.unit_complex_normal(g, (2, n)) * np.sqrt(s / (4 * OC.DF))
    return OR.to_fixed(z, frac)
