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


def test_entry_points_refuse_null_handles_without_a_gpu():
    # every status-returning call checks its handles and pointers before any CUDA work: with
    # null handles and zero sizes it returns GBK_EINVAL and names itself in the error string
    # (destroying a null network or PSD plan, and an empty mixture batch, are no-ops: GBK_OK)
    if not os.path.exists(LIB):
        pytest.skip("library not built")
    from paper_2405_04690_gb300 import _lib as L
    h = L.lib()
    no_op = {"mdn_destroy", "gbk_psd_plan_destroy", "mdn_sample_logpdf"}
    checked = 0
    for name, (res, args) in L.SIGNATURES.items():
        if res is not ctypes.c_int or name in ("gbk_version", "gmm_max_points"):
            continue
        vals = []
        for a in args:
            if a in (ctypes.c_double, ctypes.c_float):
                vals.append(0.0)
            elif a in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64):
                vals.append(0)
            else:
                vals.append(None)
        st = getattr(h, name)(*vals)
        if name in no_op:
            assert st == 0, (name, st)
        else:
            assert st == 1, (name, st)
            assert name in h.gbk_last_error().decode(), (name, h.gbk_last_error())
        checked += 1
    assert checked >= 40


def test_sizes_the_library_reports():
    # the network's parameter count is the architecture's (1024 -> 3 x 512 -> 272, weights and
    # biases), the EM point cap and the no-allocation scratch are the documented constants
    if not os.path.exists(LIB):
        pytest.skip("library not built")
    from oracle import mdn as MD
    from paper_2405_04690_gb300 import _lib as L
    assert L.lib().mdn_param_count() == MD.n_params() == 1024 * 512 + 512 + 2 * (512 * 512 + 512) + 512 * 272 + 272
    assert L.lib().gmm_max_points() == 2048
    assert L.lib().total_loglike_noalloc_capacity() == 1 << 21


def test_noalloc_binding_checks_sizes_before_the_call():
    # undersized tensors never reach the library (which would read past them): the binding
    # compares them with W and n_bins first
    torch = pytest.importorskip("torch")
    if not os.path.exists(LIB):
        pytest.skip("library not built")
    from paper_2405_04690_gb300 import _lib as L
    pp = torch.ones((4, 2), dtype=torch.float64)
    out = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError, match="residual"):
        L.total_loglike_noalloc(3.0e7, 3146, 1 << 16, torch.zeros((1, 2, 8, 2), dtype=torch.float32), pp, out)
    with pytest.raises(ValueError, match="logl"):
        L.total_loglike_noalloc(3.0e7, 3146, 8, torch.zeros((4, 2, 8, 2), dtype=torch.float32), pp, out[:2])
    with pytest.raises(ValueError, match="psd_params"):
        L.total_loglike_noalloc(3.0e7, 3146, 8, torch.zeros((4, 2, 8, 2), dtype=torch.float32), pp[:, :1], out)
