"""ctypes binding of libgbk.so (argument marshalling only).

Every function here has the name of the C entry point it calls and passes device
pointers of torch tensors straight through; all arithmetic runs in the library's
kernels. A missing library or a non-CUDA tensor raises immediately: there is no CPU
fallback.
"""
import ctypes
import math
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbk.so")

GBK_FP64 = 0
GBK_MIXED = 1
PRECISION = {"fp64": GBK_FP64, "mixed": GBK_MIXED}

STATUS = {0: "GBK_OK", 1: "GBK_EINVAL", 2: "GBK_ERANGE", 3: "GBK_ENOMEM", 4: "GBK_ECUDA",
          5: "GBK_ETIMEOUT", 6: "GBK_ENOTIMPL"}

# Every symbol the C header declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


class GbkGrid(ctypes.Structure):
    _fields_ = [("tobs", ctypes.c_double), ("dt", ctypes.c_double), ("k0", ctypes.c_int64), ("n_bins", ctypes.c_int64)]


class GbkResidual(ctypes.Structure):
    _fields_ = [("data", _vp), ("n_walkers", _i32), ("frac_bits", _i32)]


class GbkPsd(ctypes.Structure):
    _fields_ = [("params", _vp), ("n_psd", _i32)]


class GbkSweepDesc(ctypes.Structure):
    _fields_ = [("n_temps", _i32), ("n_walkers", _i32), ("n_bands", _i32), ("n_max", _i32), ("band_bins", _i32),
                ("band_k0", _i64), ("sigma", ctypes.c_double * 8), ("log_occ_odds", ctypes.c_double),
                ("props_per_source", ctypes.c_double), ("ln_a_min", ctypes.c_double), ("ln_a_max", ctypes.c_double),
                ("mc_min", ctypes.c_double), ("mc_max", ctypes.c_double), ("f_min", ctypes.c_double),
                ("f_max", ctypes.c_double), ("precision", _i32)]


class GbkPsdDesc(ctypes.Structure):
    _fields_ = [("n_temps", _i32), ("n_walkers", _i32), ("lo", ctypes.c_double * 9), ("hi", ctypes.c_double * 9),
                ("stretch_a", ctypes.c_double)]


class GbkSearchDesc(ctypes.Structure):
    _fields_ = [("n_bands", _i32), ("band_bins", _i32), ("n_temps", _i32), ("n_walkers", _i32),
                ("band_k0", ctypes.c_int64), ("ln_a_min", ctypes.c_double), ("ln_a_max", ctypes.c_double),
                ("mc_min", ctypes.c_double), ("mc_max", ctypes.c_double), ("stretch_a", ctypes.c_double),
                ("precision", _i32), ("stall_limit", _i32), ("n_sets", _i32)]


class GbkTraceRec(ctypes.Structure):
    _fields_ = [("kind", _i32), ("t", _i32), ("w", _i32), ("b", _i32), ("slot", _i32), ("seq", _i32),
                ("accepted", _i32), ("parity", _i32), ("dlogl", ctypes.c_double), ("log_alpha", ctypes.c_double),
                ("params", ctypes.c_double * 8)]


class GbkTrace(ctypes.Structure):
    _fields_ = [("records", _vp), ("capacity", _i32), ("count", _vp)]


SWEEP_INMODEL = 1
SWEEP_RJ = 2
SWEEP_SWAP = 4
SWEEP_REFRESH = 8
SWEEP_TIMING = 16
SWEEP_MDN = 32
TRACE_DTYPE_FIELDS = [("kind", "<i4"), ("t", "<i4"), ("w", "<i4"), ("b", "<i4"), ("slot", "<i4"), ("seq", "<i4"),
                      ("accepted", "<i4"), ("parity", "<i4"), ("dlogl", "<f8"), ("log_alpha", "<f8"),
                      ("params", "<f8", (8,))]

SIGNATURES = {
    "gbk_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(GbkGrid)]),
    "gbk_destroy": (ctypes.c_int, [_vp]),
    "gbk_last_error": (ctypes.c_char_p, []),
    "gbk_sync_status": (ctypes.c_int, [_vp, _vp]),
    "gbk_version": (ctypes.c_int, []),
    "gb_waveform_batch": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i64, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "gb_delta_loglike_batch": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _vp, _i64, ctypes.POINTER(GbkResidual),
                                              ctypes.POINTER(GbkPsd), _vp, ctypes.c_int, _vp]),
    "gbk_autotune_dlogl": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _vp, _i64, ctypes.POINTER(GbkResidual),
                                          ctypes.POINTER(GbkPsd), _vp, ctypes.c_int, ctypes.POINTER(_i32), _vp]),
    "residual_add_sub": (ctypes.c_int, [_vp, ctypes.POINTER(GbkResidual), _vp, _vp, _i32, _vp, _i64, _i32,
                                        ctypes.c_int, _vp]),
    "psd_eval": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "total_loglike": (ctypes.c_int, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "gbk_sweep_create": (ctypes.c_int, [_vp, ctypes.POINTER(GbkSweepDesc), ctypes.POINTER(_vp)]),
    "gbk_sweep_destroy": (ctypes.c_int, [_vp]),
    "gbk_sweep_kernel_ms": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "total_loglike_noalloc_capacity": (ctypes.c_int64, []),
    "total_loglike_noalloc": (ctypes.c_int, [ctypes.c_double, _i64, _i64, _vp, _vp, _i32, _vp, _vp]),
    "gb_sweep": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(GbkResidual), ctypes.POINTER(GbkPsd),
                                ctypes.c_uint64, ctypes.c_uint32, _i32, ctypes.POINTER(GbkTrace), _vp, _vp]),
    "mdn_param_count": (ctypes.c_int64, []),
    "mdn_create": (ctypes.c_int, [ctypes.POINTER(_vp), _i32]),
    "mdn_destroy": (ctypes.c_int, [_vp]),
    "mdn_status": (ctypes.c_int, [_vp, _vp]),
    "mdn_set_params": (ctypes.c_int, [_vp, _vp, _vp]),
    "mdn_forward": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "mdn_backward": (ctypes.c_int, [_vp, _vp, _vp, _i32, _vp, _vp, _vp]),
    "mdn_adam": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, _vp]),
    "mdn_train_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, ctypes.c_float, _vp, _vp]),
    "mdn_sample_logpdf": (ctypes.c_int, [_vp, _i32, ctypes.c_double, _vp, _vp, _vp, _vp, _i32, _vp]),
    "gmm_max_points": (_i32, []),
    "gmm_fit": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i32, ctypes.c_double, ctypes.c_double, _i32, _i32, _vp, _vp,
                               _vp, _vp]),
    "mdn_train_epoch": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, ctypes.c_float, _vp,
                                       _vp]),
    "gbk_sweep_set_proposal": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double]),
    "psd_eval_fg": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "total_loglike_fg": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp]),
    "gbk_psd_plan_create": (ctypes.c_int, [_vp, ctypes.POINTER(GbkPsdDesc), ctypes.POINTER(_vp)]),
    "gbk_psd_plan_destroy": (ctypes.c_int, [_vp]),
    "gb_psd_sweep": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_uint64, ctypes.c_uint32, _vp, _vp]),
    "gbk_search_create": (ctypes.c_int, [_vp, ctypes.POINTER(GbkSearchDesc), ctypes.POINTER(_vp)]),
    "gbk_search_destroy": (ctypes.c_int, [_vp]),
    "gb_search_init": (ctypes.c_int, [_vp, _vp, ctypes.c_uint64, ctypes.c_uint32, _vp]),
    "gb_search_windows": (ctypes.c_int, [_vp, ctypes.POINTER(GbkResidual), _i32, _vp]),
    "gb_search_eval": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(GbkPsd), _i32, _vp]),
    "gb_search_sweep": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(GbkPsd), _i32, ctypes.c_uint64,
                                       ctypes.c_uint32, _vp, _vp, _vp, _vp, _vp]),
    "gb_search_samples": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _vp, _i32,
                                         _i32, _vp]),
    "gb_search_ball": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, _vp]),
    "gbk_sweep_adapt_temps": (ctypes.c_int, [_vp, _vp, _i32, ctypes.c_double, ctypes.c_double, _vp]),
    "gbk_sweep_transfer": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gbk_sweep_update_group": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _i32, _vp]),
    "gb_sweep_features": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(GbkResidual), ctypes.POINTER(GbkPsd), _vp, _vp,
                                         _vp]),
}

_LIB = None


class GbkError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib().gbk_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), msg))


def lib():
    """Load libgbk.so (once); raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgbk.so is not built (%s); run python -m paper_2405_04690_gb300.build" % LIB_PATH)
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = h
    return _LIB


def _check(status, where):
    if status != 0:
        raise GbkError(status, where)


def _dev(t, dtype, name, writable=False):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns a gbk_ctx (orbit/twiddle/PSD tables and scratch on the current device)."""

    def __init__(self, tobs, dt, k0, n_bins):
        self.grid = GbkGrid(float(tobs), float(dt), int(k0), int(n_bins))
        h = _vp()
        _check(lib().gbk_create(ctypes.byref(h), ctypes.byref(self.grid)), "gbk_create")
        self.handle = h

    @property
    def k0(self):
        return self.grid.k0

    @property
    def n_bins(self):
        return self.grid.n_bins

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().gbk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gbk_sync_status(ctx, stream=None):
    """Synchronise the stream and raise GbkError if a kernel set the context's error word."""
    _check(lib().gbk_sync_status(ctx.handle, _stream(stream)), "gbk_sync_status")


def gb_waveform_batch(ctx, params, n_band, n_band_max, k_start, h_a, h_e, out_off, precision, stream=None):
    """TDI A/E bands of n sources (Sec. II.A, App. F): params [8][n] float64, n_band [n] int32,
    k_start [n] int64 out, h_a / h_e packed complex bands out (complex64 for GBK_MIXED,
    complex128 for GBK_FP64; source i at element out_off[i], out_off [n] int64)."""
    n = params.shape[1]
    cdt = torch.complex64 if precision == GBK_MIXED else torch.complex128
    _check(lib().gb_waveform_batch(ctx.handle, _dev(params, torch.float64, "params"), _dev(n_band, torch.int32, "n_band"),
                                   int(n_band_max), n, _dev(k_start, torch.int64, "k_start"),
                                   _dev(h_a, cdt, "h_a"), _dev(h_e, cdt, "h_e"), _dev(out_off, torch.int64, "out_off"),
                                   int(precision), _stream(stream)), "gb_waveform_batch")


def residual_struct(resid, frac_bits):
    """gbk_residual for an int64 tensor [W][2][n_bins][2]. The struct keeps a reference to the
    tensor: it holds the tensor's device address, which must stay allocated while the struct
    (or work queued with it) is in use."""
    _dev(resid, torch.int64, "residual")
    s = GbkResidual(ctypes.c_void_p(resid.data_ptr()), int(resid.shape[0]), int(frac_bits))
    s._tensor = resid
    return s


def psd_struct(psd_params):
    """gbk_psd for a float64 tensor [n_psd][2] (the struct keeps a reference to the tensor)."""
    _dev(psd_params, torch.float64, "psd_params")
    s = GbkPsd(ctypes.c_void_p(psd_params.data_ptr()), int(psd_params.shape[0]))
    s._tensor = psd_params
    return s


def gb_delta_loglike_batch(ctx, params_new, params_old, n_band, n_band_max, walker, residual, psd, dlogl,
                           precision, stream=None):
    """Delta lnL of n independent swaps old -> new (Eq. swapsource; amplitude 0 old: birth, new: death)
    against walker[i]'s residual: params_* [8][n] float64, n_band / walker [n] int32, residual from
    residual_struct, psd from psd_struct, dlogl [n] float64 out."""
    n = params_new.shape[1]
    _check(lib().gb_delta_loglike_batch(ctx.handle, _dev(params_new, torch.float64, "params_new"),
                                        _dev(params_old, torch.float64, "params_old"), _dev(n_band, torch.int32, "n_band"),
                                        int(n_band_max), _dev(walker, torch.int32, "walker"), n,
                                        ctypes.byref(residual), ctypes.byref(psd), _dev(dlogl, torch.float64, "dlogl"),
                                        int(precision), _stream(stream)), "gb_delta_loglike_batch")


def residual_add_sub(ctx, residual, params, n_band, n_band_max, walker, sign, precision, stream=None):
    """sign +1: the sources enter the model (R <- R - h); -1: they leave (R <- R + h); bit-exact inverse
    pair on the int64 fixed-point residual. params [8][n] float64, n_band / walker [n] int32."""
    n = params.shape[1]
    _check(lib().residual_add_sub(ctx.handle, ctypes.byref(residual), _dev(params, torch.float64, "params"),
                                  _dev(n_band, torch.int32, "n_band"), int(n_band_max), _dev(walker, torch.int32, "walker"),
                                  n, int(sign), int(precision), _stream(stream)), "residual_add_sub")


def psd_eval(ctx, psd_params, s_out, stream=None):
    """Eq. psd on the context window: psd_params [W][2] float64 (sqrt S_oms, sqrt S_acc), s_out
    [W][n_bins] float64 out (or None)."""
    w = psd_params.shape[0]
    _check(lib().psd_eval(ctx.handle, _dev(psd_params, torch.float64, "psd_params"), w,
                          _dev(s_out, torch.float64, "s_out") if s_out is not None else None, _stream(stream)), "psd_eval")


def total_loglike(ctx, residual, psd_params, logl, stream=None):
    """Eq. like per walker: residual [W][2][n_bins][2] float32, psd_params [W][2] float64, logl [W]
    float64 out."""
    w = psd_params.shape[0]
    _check(lib().total_loglike(ctx.handle, _dev(residual, torch.float32, "residual"),
                               _dev(psd_params, torch.float64, "psd_params"), w, _dev(logl, torch.float64, "logl"),
                               _stream(stream)), "total_loglike")


class SweepPlan:
    """Owns a gbk_sweep (residual snapshot, opened windows, waveform cache)."""

    def __init__(self, ctx, n_temps, n_walkers, n_bands, n_max, band_bins, band_k0, sigma, precision,
                 log_occ_odds=0.0, props_per_source=1.0, ln_a_min=None, ln_a_max=None, mc_min=0.3, mc_max=0.8,
                 f_min=1e-3, f_max=4e-3):
        d = GbkSweepDesc()
        d.n_temps, d.n_walkers, d.n_bands, d.n_max, d.band_bins = n_temps, n_walkers, n_bands, n_max, band_bins
        d.band_k0 = int(band_k0)
        for i in range(8):
            d.sigma[i] = float(sigma[i])
        d.log_occ_odds = float(log_occ_odds)
        d.props_per_source = float(props_per_source)
        d.ln_a_min = math.log(1e-23) if ln_a_min is None else float(ln_a_min)
        d.ln_a_max = math.log(10 ** -21.5) if ln_a_max is None else float(ln_a_max)
        d.mc_min, d.mc_max, d.f_min, d.f_max = float(mc_min), float(mc_max), float(f_min), float(f_max)
        d.precision = int(precision)
        self.desc = d
        self.ctx = ctx
        h = _vp()
        _check(lib().gbk_sweep_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)), "gbk_sweep_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().gbk_sweep_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gb_sweep(plan, params, exists, betas, residual, psd, key, sweep_index, flags, trace=None, stats=None, stream=None):
    """One sweep of the ensemble (in-model moves, flip-all RJ, tempering swaps per the flags):
    params [T][W][B][n_max][8] float64 and exists [T][W][B][n_max] uint8 in/out, betas [B][T]
    float64, residual / psd structs, stats [5][2] int64 (added to) or None.
    trace: (records uint8 tensor of capacity*sizeof(GbkTraceRec) bytes, capacity, count int32 tensor) or None."""
    tr = None
    if trace is not None:
        rec, cap, cnt = trace
        tr = GbkTrace(ctypes.c_void_p(rec.data_ptr()), int(cap), ctypes.c_void_p(cnt.data_ptr()))
    _check(lib().gb_sweep(plan.handle, _dev(params, torch.float64, "params"), _dev(exists, torch.uint8, "exists"),
                          _dev(betas, torch.float64, "betas"), ctypes.byref(residual), ctypes.byref(psd),
                          ctypes.c_uint64(int(key)), ctypes.c_uint32(int(sweep_index)), int(flags),
                          ctypes.byref(tr) if tr is not None else None,
                          _dev(stats, torch.int64, "stats") if stats is not None else None, _stream(stream)), "gb_sweep")


def gbk_sweep_kernel_ms(plan):
    """Per-kernel device ms of the last timed sweep: (refresh, open, band, swap)."""
    out = (ctypes.c_double * 4)()
    _check(lib().gbk_sweep_kernel_ms(plan.handle, out), "gbk_sweep_kernel_ms")
    return list(out)


def total_loglike_noalloc(tobs, k0, n_bins, residual, psd_params, logl, stream=None):
    """Total log-likelihood of W walkers without a context and without allocating (fixed scratch).

    residual [W][2][n_bins][2] float32, psd_params [W][2] float64, logl [W] float64 (out);
    the sizes are checked here, before the library reads any of them."""
    if psd_params.dim() != 2 or psd_params.shape[1] != 2:
        raise ValueError("total_loglike_noalloc: psd_params must be [W][2]")
    w = psd_params.shape[0]
    if residual.numel() < 4 * w * int(n_bins):
        raise ValueError("total_loglike_noalloc: residual holds %d floats, [W][2][n_bins][2] needs %d"
                         % (residual.numel(), 4 * w * int(n_bins)))
    if logl.numel() < w:
        raise ValueError("total_loglike_noalloc: logl holds %d entries, W = %d" % (logl.numel(), w))
    _check(lib().total_loglike_noalloc(float(tobs), int(k0), int(n_bins), _dev(residual, torch.float32, "residual"),
                                       _dev(psd_params, torch.float64, "psd_params"), w,
                                       _dev(logl, torch.float64, "logl"), _stream(stream)), "total_loglike_noalloc")


def gbk_autotune_dlogl(ctx, params_new, params_old, n_band, n_band_max, walker, residual, psd, dlogl, precision,
                       stream=None):
    """Autotune the Delta lnL launch shape for one band length; returns (warps/CTA, CTAs/SM)."""
    n = params_new.shape[1]
    best = (_i32 * 2)()
    _check(lib().gbk_autotune_dlogl(ctx.handle, _dev(params_new, torch.float64, "params_new"),
                                    _dev(params_old, torch.float64, "params_old"), _dev(n_band, torch.int32, "n_band"),
                                    int(n_band_max), _dev(walker, torch.int32, "walker"), n, ctypes.byref(residual),
                                    ctypes.byref(psd), _dev(dlogl, torch.float64, "dlogl"), int(precision), best,
                                    _stream(stream)), "gbk_autotune_dlogl")
    return int(best[0]), int(best[1])


# ------------------------------------------------------------------ learned proposal
class Mdn:
    """Owns a gbk_mdn workspace (BF16 weight copy, activations, gradient partials)."""

    def __init__(self, max_batch):
        h = _vp()
        _check(lib().mdn_create(ctypes.byref(h), int(max_batch)), "mdn_create")
        self.handle = h
        self.max_batch = int(max_batch)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().mdn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mdn_status(net, stream=None):
    """Synchronise and raise GbkError if a tensor-core product of the workspace gave up a wait."""
    _check(lib().mdn_status(net.handle, _stream(stream)), "mdn_status")


def mdn_param_count():
    """Length of the flat float32 parameter vector (W1 b1 W2 b2 W3 b3 W4 b4)."""
    return int(lib().mdn_param_count())


def mdn_set_params(net, params, stream=None):
    """Load float32 parameters [mdn_param_count()] into the workspace's BF16 copies."""
    _check(lib().mdn_set_params(net.handle, _dev(params, torch.float32, "params"), _stream(stream)), "mdn_set_params")


def mdn_forward(net, x, raw, stream=None):
    """raw [B][272] float32 = network(x), x [B][1024] bfloat16."""
    _check(lib().mdn_forward(net.handle, _dev(x, torch.bfloat16, "x"), int(x.shape[0]), _dev(raw, torch.float32, "raw"),
                             _stream(stream)), "mdn_forward")


def mdn_backward(net, x, u, grad, loss=None, stream=None):
    """grad [mdn_param_count()] float32 = d(mean -ln q(u | x))/d(params); x [B][1024] bfloat16,
    u [B][8] float32 unit coordinates; loss (float64 [1] or None) out."""
    _check(lib().mdn_backward(net.handle, _dev(x, torch.bfloat16, "x"), _dev(u, torch.float32, "u"), int(x.shape[0]),
                              _dev(grad, torch.float32, "grad"),
                              _dev(loss, torch.float64, "loss") if loss is not None else None, _stream(stream)),
           "mdn_backward")


def mdn_adam(net, params, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step on the caller's float32 params / moments (step counts from 1)."""
    _check(lib().mdn_adam(net.handle, _dev(params, torch.float32, "params"), _dev(m, torch.float32, "m"),
                          _dev(v, torch.float32, "v"), _dev(grad, torch.float32, "grad"), int(step), float(lr),
                          float(beta1), float(beta2), float(eps), _stream(stream)), "mdn_adam")


def mdn_train_step(net, params, m, v, x, u, step, lr, loss=None, stream=None):
    """mdn_backward then Adam on one batch, the gradient kept on the device."""
    _check(lib().mdn_train_step(net.handle, _dev(params, torch.float32, "params"), _dev(m, torch.float32, "m"),
                                _dev(v, torch.float32, "v"), _dev(x, torch.bfloat16, "x"), _dev(u, torch.float32, "u"),
                                int(x.shape[0]), int(step), float(lr),
                                _dev(loss, torch.float64, "loss") if loss is not None else None, _stream(stream)),
           "mdn_train_step")


def mdn_train_epoch(net, params, m, v, x, u, order, batch, step0, lr, loss=None, stream=None):
    """len(order) // batch Adam steps over rows of x [n][1024] bf16 / u [n][8] picked by order (int32, device)."""
    n_steps = int(order.numel()) // int(batch)
    _check(lib().mdn_train_epoch(net.handle, _dev(params, torch.float32, "params"), _dev(m, torch.float32, "m"),
                                 _dev(v, torch.float32, "v"), _dev(x, torch.bfloat16, "x"), _dev(u, torch.float32, "u"),
                                 int(x.shape[0]), _dev(order, torch.int32, "order"), int(batch), n_steps, int(step0),
                                 float(lr), _dev(loss, torch.float64, "loss") if loss is not None else None,
                                 _stream(stream)), "mdn_train_epoch")
    return n_steps


def mdn_sample_logpdf(raw, eps, precision, words=None, u_out=None, u_in=None, logq=None, stream=None):
    """Draws (words [B][9] int32 bit patterns -> u_out [B][8]) from, or densities (u_in [B][8]) of, the
    eps-defensive truncated mixture of raw [B][272]; logq [B] float32 out."""
    _check(lib().mdn_sample_logpdf(_dev(raw, torch.float32, "raw"), int(raw.shape[0]), float(eps),
                                   _dev(words, torch.int32, "words") if words is not None else None,
                                   _dev(u_out, torch.float32, "u_out") if u_out is not None else None,
                                   _dev(u_in, torch.float32, "u_in") if u_in is not None else None,
                                   _dev(logq, torch.float32, "logq") if logq is not None else None,
                                   int(precision), _stream(stream)), "mdn_sample_logpdf")


def gmm_max_points():
    """Most present points per group that gmm_fit uses (the first ones)."""
    return int(lib().gmm_max_points())


def gmm_fit(x, raw_out, n_comp=16, n_iter=50, reg=1e-6, min_weight=0.01, precision=GBK_MIXED, fit_out=None,
            loglike=None, stream=None):
    """Batched EM fit of x [G][P][8] (float32, NaN rows absent); raw_out [C][G][272] float32."""
    if x.dim() != 3 or x.shape[2] != 8 or raw_out.dim() != 3 or raw_out.shape[1:] != (x.shape[0], 272):
        raise ValueError("gmm_fit: x must be [G][P][8] and raw_out [C][G][272]")
    _check(lib().gmm_fit(_dev(x, torch.float32, "x"), int(x.shape[0]), int(x.shape[1]), int(n_comp), int(n_iter),
                         float(reg), float(min_weight), int(precision), int(raw_out.shape[0]),
                         _dev(raw_out, torch.float32, "raw_out"), _dev(fit_out, torch.float64, "fit_out"),
                         _dev(loglike, torch.float64, "loglike"), _stream(stream)), "gmm_fit")


def gbk_sweep_set_proposal(plan, net=None, raw_table=None, eps=0.1, inmodel_frac=0.0):
    """Attach the learned proposal (a network, or a fixed raw table [W][n_bands][272]) to a sweep plan."""
    plan._proposal_refs = (net, raw_table)   # keep them alive while the plan uses them
    _check(lib().gbk_sweep_set_proposal(plan.handle, net.handle if net is not None else None,
                                        _dev(raw_table, torch.float32, "raw_table") if raw_table is not None else None,
                                        float(eps), float(inmodel_frac)), "gbk_sweep_set_proposal")


def gbk_sweep_adapt_temps(plan, betas, iteration, nu=100.0, t0=1000.0, stream=None):
    """Adapt every band's ladder from the last sweep's swap acceptance (in place)."""
    _check(lib().gbk_sweep_adapt_temps(plan.handle, _dev(betas, torch.float64, "betas"), int(iteration), float(nu),
                                       float(t0), _stream(stream)), "gbk_sweep_adapt_temps")


def gbk_sweep_transfer(plan, params, exists, counts=None, stream=None):
    """Band-edge ownership transfer of the cold chain (in place); counts: optional int32[2]
    device tensor to which (moved, blocked) are added."""
    _check(lib().gbk_sweep_transfer(plan.handle, _dev(params, torch.float64, "params"),
                                    _dev(exists, torch.uint8, "exists"),
                                    None if counts is None else _dev(counts, torch.int32, "counts"),
                                    _stream(stream)), "gbk_sweep_transfer")


def gbk_sweep_update_group(plan, params, exists, frac, n_friends=32, stream=None):
    """Rebuild every band's stationary group from the cold chain; frac of in-model moves become group stretches."""
    _check(lib().gbk_sweep_update_group(plan.handle, _dev(params, torch.float64, "params"),
                                        _dev(exists, torch.uint8, "exists"), float(frac), int(n_friends),
                                        _stream(stream)), "gbk_sweep_update_group")


def gb_sweep_features(plan, params, exists, residual, psd, x_out=None, u_out=None, stream=None):
    """Features [W][n_bands][1024] bfloat16 and cold-slot unit coordinates [W][n_bands][n_max][8] float32."""
    _check(lib().gb_sweep_features(plan.handle, _dev(params, torch.float64, "params"),
                                   _dev(exists, torch.uint8, "exists"), ctypes.byref(residual), ctypes.byref(psd),
                                   _dev(x_out, torch.bfloat16, "x_out") if x_out is not None else None,
                                   _dev(u_out, torch.float32, "u_out") if u_out is not None else None,
                                   _stream(stream)), "gb_sweep_features")


# ------------------------------------------------------------------ noise PSD and foreground
def psd_eval_fg(ctx, psd_params, s_out, stream=None):
    """Per-channel PSD [W][2][n_bins] float64 of the 9-parameter model."""
    _check(lib().psd_eval_fg(ctx.handle, _dev(psd_params, torch.float64, "psd_params"), int(psd_params.shape[0]),
                             _dev(s_out, torch.float64, "s_out") if s_out is not None else None, _stream(stream)),
           "psd_eval_fg")


def total_loglike_fg(ctx, residual, psd_params, logl, resid_index=None, stream=None):
    """Eq. like for entries psd_params [n][9] against residual [n_resid][2][n_bins][2] float32."""
    _check(lib().total_loglike_fg(ctx.handle, _dev(residual, torch.float32, "residual"), int(residual.shape[0]),
                                  _dev(psd_params, torch.float64, "psd_params"),
                                  _dev(resid_index, torch.int32, "resid_index") if resid_index is not None else None,
                                  int(psd_params.shape[0]), _dev(logl, torch.float64, "logl"), _stream(stream)),
           "total_loglike_fg")


class PsdPlan:
    """Owns a gbk_psd_plan (proposal buffers and partial sums of the PSD sampler)."""

    def __init__(self, ctx, n_temps, n_walkers, lo, hi, stretch_a=2.0):
        d = GbkPsdDesc()
        d.n_temps, d.n_walkers = int(n_temps), int(n_walkers)
        for i in range(9):
            d.lo[i], d.hi[i] = float(lo[i]), float(hi[i])
        d.stretch_a = float(stretch_a)
        self.desc = d
        h = _vp()
        _check(lib().gbk_psd_plan_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)), "gbk_psd_plan_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().gbk_psd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gb_psd_sweep(plan, params, logl, residual, betas, key, sweep_index, stats=None, stream=None):
    _check(lib().gb_psd_sweep(plan.handle, _dev(params, torch.float64, "params"), _dev(logl, torch.float64, "logl"),
                              _dev(residual, torch.float32, "residual"), _dev(betas, torch.float64, "betas"),
                              ctypes.c_uint64(int(key)), ctypes.c_uint32(int(sweep_index)),
                              _dev(stats, torch.int64, "stats") if stats is not None else None, _stream(stream)),
           "gb_psd_sweep")


class SearchPlan:
    """Owns a gbk_search plan (per-band search sampler of the search-RJ proposal)."""

    def __init__(self, ctx, n_bands, band_bins, band_k0, n_temps, n_walkers, precision=GBK_MIXED,
                 ln_a_min=math.log(1e-23), ln_a_max=math.log(10 ** -21.5), mc_min=0.3, mc_max=0.8, stretch_a=2.0,
                 stall_limit=0, n_sets=1):
        d = GbkSearchDesc()
        d.n_bands, d.band_bins, d.n_temps, d.n_walkers = int(n_bands), int(band_bins), int(n_temps), int(n_walkers)
        d.band_k0 = int(band_k0)
        d.ln_a_min, d.ln_a_max, d.mc_min, d.mc_max = float(ln_a_min), float(ln_a_max), float(mc_min), float(mc_max)
        d.stretch_a = float(stretch_a)
        d.precision = int(precision)
        d.stall_limit = int(stall_limit)
        d.n_sets = int(n_sets)
        self.desc = d
        h = _vp()
        _check(lib().gbk_search_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)), "gbk_search_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().gbk_search_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gb_search_init(plan, u, key, seed, stream=None):
    _check(lib().gb_search_init(plan.handle, _dev(u, torch.float64, "u"), ctypes.c_uint64(int(key)),
                                ctypes.c_uint32(int(seed)), _stream(stream)), "gb_search_init")


def gb_search_windows(plan, residual, walker, stream=None):
    _check(lib().gb_search_windows(plan.handle, ctypes.byref(residual), int(walker), _stream(stream)),
           "gb_search_windows")


def gb_search_eval(plan, u, ell, psd, psd_walker=0, stream=None):
    _check(lib().gb_search_eval(plan.handle, _dev(u, torch.float64, "u"), _dev(ell, torch.float64, "ell"),
                                ctypes.byref(psd), int(psd_walker), _stream(stream)), "gb_search_eval")


def gb_search_sweep(plan, u, ell, betas, psd, key, sweep_index, psd_walker=0, best=None, stats=None, stream=None):
    """best: (best_ell [B] float64, best_u [B][8] float64, stall [B] int32) or None."""
    be, bu, st = best if best is not None else (None, None, None)
    _check(lib().gb_search_sweep(plan.handle, _dev(u, torch.float64, "u"), _dev(ell, torch.float64, "ell"),
                                 _dev(betas, torch.float64, "betas"), ctypes.byref(psd), int(psd_walker),
                                 ctypes.c_uint64(int(key)), ctypes.c_uint32(int(sweep_index)),
                                 _dev(be, torch.float64, "best_ell"), _dev(bu, torch.float64, "best_u"),
                                 _dev(st, torch.int32, "stall"), _dev(stats, torch.int64, "stats"), _stream(stream)),
           "gb_search_sweep")


def gb_search_samples(plan, u, best_ell, snr_min, f_min, f_max, x, row0, stream=None):
    """Cold walkers of every band into x [n_sets][n_bands][n_rows][8] or [n_sets n_bands][n_rows][8]
    (float32) at rows row0 .. row0 + W."""
    _check(lib().gb_search_samples(plan.handle, _dev(u, torch.float64, "u"), _dev(best_ell, torch.float64, "best_ell"),
                                   float(snr_min), float(f_min), float(f_max), _dev(x, torch.float32, "x"),
                                   int(x.shape[-2]), int(row0), _stream(stream)), "gb_search_samples")


def gb_search_ball(plan, u, best_ell, best_u, sigma, key, seed, stream=None):
    """Walkers of bands with a best point redrawn around it (clipped normal of width sigma)."""
    _check(lib().gb_search_ball(plan.handle, _dev(u, torch.float64, "u"), _dev(best_ell, torch.float64, "best_ell"),
                                _dev(best_u, torch.float64, "best_u"), float(sigma), ctypes.c_uint64(int(key)),
                                ctypes.c_uint32(int(seed)), _stream(stream)), "gb_search_ball")
