"""The C ABI library loads and exports every function include/gbk.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbk.h")
LIB = os.path.join(ROOT, "paper_2405_04690_gb300", "libgbk.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:gbk_status|const char\*|int|int32_t|int64_t)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for want in ("gb_waveform_batch", "gb_delta_loglike_batch", "residual_add_sub", "psd_eval", "total_loglike"):
        assert want in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(LIB):
        from paper_2405_04690_gb300 import build
        build.build()
    h = ctypes.CDLL(LIB)
    missing = [n for n in declared_functions() if not hasattr(h, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2405_04690_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_version_and_error_string_without_gpu():
    if not os.path.exists(LIB):
        pytest.skip("library not built")
    h = ctypes.CDLL(LIB)
    h.gbk_version.restype = ctypes.c_int
    h.gbk_last_error.restype = ctypes.c_char_p
    assert h.gbk_version() >= 100
    assert isinstance(h.gbk_last_error(), bytes)


def test_binding_refuses_host_tensors():
    # the product path has no CPU fallback: host tensors are refused before any library call
    torch = pytest.importorskip("torch")
    from paper_2405_04690_gb300 import _lib as L
    x = torch.zeros((2, 16, 8), dtype=torch.float32)
    raw = torch.zeros((1, 2, 272), dtype=torch.float32)
    with pytest.raises(TypeError, match="CUDA tensor"):
        L.gmm_fit(x, raw)
    with pytest.raises(TypeError, match="CUDA tensor"):
        L.psd_struct(torch.zeros((1, 2), dtype=torch.float64))
