"""Thin ctypes binding of ``libhist.so`` (the C ABI in ``include/hist.h``).

Argument marshalling only: every step of the fill runs in the library's CUDA
kernels.  There is no CPU fallback -- if ``libhist.so`` is missing or cannot
be loaded, every call raises.  PyTorch is used for device memory and the
current stream (``data_ptr()``, ``torch.cuda.current_stream().cuda_stream``).

The functions keep the C names (``hist_book``, ``hist_fill_bulk``,
``hist_result`` ...); :class:`Hist` is a small owner object around them.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhist.so")

HIST_OK = 0
HIST_ERR_ARG = -1
HIST_ERR_AXIS = -2
HIST_ERR_CUDA = -3
HIST_ERR_OOM = -4
HIST_ERR_ALIGN = -5
HIST_ERR_TIMEOUT = -6
HIST_ERR_LOCATOR = -7
HIST_ERR_STATE = -8
HIST_ERR_UNSUPPORTED = -9
HIST_ERR_TOO_LARGE = -10

HIST_AXIS_FIXED = 0
HIST_AXIS_VARIABLE = 1

HIST_TRACK_COUNTS = 1 << 0
HIST_STAT_OVERFLOWS = 1 << 1
HIST_SUMW2 = 1 << 2
HIST_STATS_EXACT = 1 << 3
HIST_PREC_FP64 = 0 << 4
HIST_PREC_FP32C = 1 << 4
HIST_PREC_F64ATOMIC = 2 << 4
HIST_LOCATOR_AUTO = 0 << 8
HIST_LOCATOR_LEARNED = 1 << 8
HIST_LOCATOR_BSEARCH = 2 << 8


class HistError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class hist_locator_opts_t(ctypes.Structure):
    _fields_ = [("segments", ctypes.c_int32), ("steps", ctypes.c_int32), ("lr", ctypes.c_float),
                ("apply", ctypes.c_int32)]


class hist_locator_report_t(ctypes.Structure):
    _fields_ = [("segments", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("window_untrained", ctypes.c_int32), ("window", ctypes.c_int32),
                ("loss_untrained", ctypes.c_double), ("loss", ctypes.c_double),
                ("train_ms", ctypes.c_double)]


class hist_define_t(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32)]


class hist_filter_t(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int32), ("op", ctypes.c_int32), ("value", ctypes.c_double)]


HIST_DEF_COL, HIST_DEF_SUMSQ, HIST_DEF_HYPOT, HIST_DEF_MUL, HIST_DEF_ADD, HIST_DEF_SUB = range(6)
HIST_FLT_NE, HIST_FLT_EQ, HIST_FLT_LT, HIST_FLT_LE, HIST_FLT_GT, HIST_FLT_GE = range(6)


class hist_batch_tuning_t(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("smem_hists", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("worst_ms", ctypes.c_double),
                ("strategy", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("replicas", ctypes.c_int32), ("cost_cap_tenths", ctypes.c_int32),
                ("events_per_thread", ctypes.c_int32)]


HIST_BATCH_GRAPH = 1 << 0
HIST_BATCH_WIDE = 1 << 1
HIST_BATCH_SLICED = 1 << 2


class hist_axis_t(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nbins", ctypes.c_int32),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("edges", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p


def load(path: str | None = None):
    """Load libhist.so (raises if it is not built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_2401_13310_gb300.build()")
        lib = ctypes.CDLL(p)
        sig = {
            "hist_book": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint32, _P]),
            "hist_fill_bulk": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
            "hist_result": (ctypes.c_int, [_P, _P, _P]),
            "hist_counts": (ctypes.c_int, [_P, _P]),
            "hist_locate": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
            "hist_reset": (ctypes.c_int, [_P]),
            "hist_free": (None, [_P]),
            "hist_nbins_total": (ctypes.c_int64, [_P]),
            "hist_nstats": (ctypes.c_int, [_P]),
            "hist_ndim": (ctypes.c_int, [_P]),
            "hist_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "hist_version": (ctypes.c_char_p, []),
            "hist_axis_thresholds": (ctypes.c_int, [_P, _P]),
            "hist_axis_affine": (ctypes.c_int, [_P, _P, _P, _P]),
            "hist_fill_bulk_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_uint32, _P, _P, _P]),
            "hist_train_locator": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
            "hist_batch_create": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_uint32, _P]),
            "hist_batch_fill": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int64, _P]),
            "hist_batch_tune": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int64, _P]),
            "hist_set_kernel_timing": (ctypes.c_int, [_P, ctypes.c_int]),
            "hist_sumw2": (ctypes.c_int, [_P, _P]),
            "hist_fill_columns": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.c_int, _P, ctypes.c_int64,
                                                 _P]),
            "hist_fill_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int64, _P]),
            "hist_locator_mode": (ctypes.c_int, [_P, ctypes.c_int]),
            "hist_kernel_time": (ctypes.c_int, [_P, _P, _P]),
            "hist_batch_configure": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]),
            "hist_batch_free": (None, [_P]),
            "hist_locator_loss_grad": (ctypes.c_int, [ctypes.c_int, ctypes.c_float, ctypes.c_float, _P, _P, _P,
                                                      _P, ctypes.c_int64, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().hist_strerror(code).decode()
    except Exception:  # pragma: no cover - only when the library is absent
        return "status"


def _check(code: int, where: str) -> None:
    if code != HIST_OK:
        raise HistError(code, where)


def make_axes(axes):
    """Plain axis dicts -> (ctypes array, keepalive)."""
    arr = (hist_axis_t * len(axes))()
    keep = []
    for d, ax in enumerate(axes):
        if ax["kind"] == "fixed":
            arr[d].kind = HIST_AXIS_FIXED
            arr[d].nbins = int(ax["nbins"])
            arr[d].xmin = float(ax["xmin"])
            arr[d].xmax = float(ax["xmax"])
            arr[d].edges = None
        else:
            e = np.ascontiguousarray(ax["edges"], dtype=np.float64)
            keep.append(e)
            arr[d].kind = HIST_AXIS_VARIABLE
            arr[d].nbins = int(e.shape[0] - 1)
            arr[d].edges = e.ctypes.data
    return arr, keep


def _ptr(x) -> int | None:
    """Device/host address of a torch tensor, numpy array or raw int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- C names ----

def hist_book(axes, flags: int = 0) -> int:
    arr, keep = make_axes(axes)
    out = ctypes.c_void_p()
    rc = load().hist_book(ctypes.addressof(arr), len(axes), int(flags), ctypes.byref(out))
    del keep
    _check(rc, "hist_book")
    return out.value


def hist_fill_bulk(h: int, values, weights, n: int, stream=None) -> None:
    _check(load().hist_fill_bulk(h, _ptr(values), _ptr(weights), int(n), _stream_ptr(stream)),
           "hist_fill_bulk")


def hist_locate(h: int, values, n: int, out, stream=None) -> None:
    _check(load().hist_locate(h, _ptr(values), int(n), _ptr(out), _stream_ptr(stream)), "hist_locate")


def hist_nbins_total(h: int) -> int:
    return int(load().hist_nbins_total(h))


def hist_nstats(h: int) -> int:
    return int(load().hist_nstats(h))


def hist_result(h: int):
    nb, ns = hist_nbins_total(h), hist_nstats(h)
    bins = np.zeros(nb, dtype=np.float64)
    stats = np.zeros(ns, dtype=np.float64)
    _check(load().hist_result(h, bins.ctypes.data, stats.ctypes.data), "hist_result")
    return bins, stats


def hist_counts(h: int) -> np.ndarray:
    c = np.zeros(hist_nbins_total(h), dtype=np.uint64)
    _check(load().hist_counts(h, c.ctypes.data), "hist_counts")
    return c


def hist_reset(h: int) -> None:
    _check(load().hist_reset(h), "hist_reset")


def hist_free(h: int) -> None:
    load().hist_free(h)


def hist_axis_thresholds(axis) -> np.ndarray:
    """The exact threshold keys (int64, nbins + 3) the device compares against."""
    arr, keep = make_axes([axis])
    nb = int(arr[0].nbins)
    out = np.zeros(nb + 3, dtype=np.int64)
    rc = load().hist_axis_thresholds(ctypes.addressof(arr), out.ctypes.data)
    del keep
    _check(rc, "hist_axis_thresholds")
    return out


def hist_axis_affine(axis):
    """(scale, offset, eps) of the FP32 estimate a fixed axis is located
    with, or None when the axis is located by its thresholds alone."""
    arr, keep = make_axes([axis])
    s, o, e = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    rc = load().hist_axis_affine(ctypes.addressof(arr), ctypes.byref(s), ctypes.byref(o), ctypes.byref(e))
    del keep
    if rc == HIST_ERR_UNSUPPORTED:
        return None
    _check(rc, "hist_axis_affine")
    return s.value, o.value, e.value


def hist_fill_bulk_noalloc(axis, values, weights, n: int, flags: int, bins_out, stats_out,
                           stream=None) -> None:
    """Allocation-free 1D fill into caller-owned device outputs (see hist.h)."""
    arr, keep = make_axes([axis])
    rc = load().hist_fill_bulk_noalloc(ctypes.addressof(arr), _ptr(values), _ptr(weights), int(n),
                                       int(flags), _ptr(bins_out), _ptr(stats_out), _stream_ptr(stream))
    del keep
    _check(rc, "hist_fill_bulk_noalloc")


def hist_train_locator(h: int, axis: int, segments: int = 0, steps: int = 0, lr: float = 0.0,
                       apply: bool = True) -> dict:
    """Train, certify and (apply) install the learned locator of one variable axis."""
    o = hist_locator_opts_t(int(segments), int(steps), float(lr), 1 if apply else 0)
    r = hist_locator_report_t()
    _check(load().hist_train_locator(h, int(axis), ctypes.byref(o), ctypes.byref(r)), "hist_train_locator")
    return {f: getattr(r, f) for f, _ in hist_locator_report_t._fields_}


def hist_locator_loss_grad(nseg: int, u0: float, u_scale: float, base, theta, x, target):
    """GPU loss and gradient of the locator's training objective (host arrays)."""
    base = np.ascontiguousarray(base, dtype=np.int32)
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    target = np.ascontiguousarray(target, dtype=np.float32)
    grad = np.zeros(nseg + 1, dtype=np.float32)
    loss = ctypes.c_double()
    _check(load().hist_locator_loss_grad(int(nseg), float(u0), float(u_scale), base.ctypes.data,
                                         theta.ctypes.data, x.ctypes.data, target.ctypes.data, x.shape[0],
                                         ctypes.byref(loss), grad.ctypes.data), "hist_locator_loss_grad")
    return loss.value, grad


def _col_array(cols):
    arr = (ctypes.c_void_p * len(cols))()
    for i, c in enumerate(cols):
        arr[i] = _ptr(c)
    return arr


def hist_batch_create(hists, col_of_hist, flags: int = 0) -> int:
    hs = (ctypes.c_void_p * len(hists))(*[int(h) for h in hists])
    cols = np.ascontiguousarray(col_of_hist, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(load().hist_batch_create(hs, len(hists), cols.ctypes.data, int(flags), ctypes.byref(out)),
           "hist_batch_create")
    return out.value


def hist_batch_fill(b: int, cols, weights, n: int, stream=None) -> None:
    arr = _col_array(cols)
    _check(load().hist_batch_fill(b, arr, len(cols), _ptr(weights), int(n), _stream_ptr(stream)),
           "hist_batch_fill")


def hist_batch_tune(b: int, cols, weights, n: int) -> dict:
    arr = _col_array(cols)
    r = hist_batch_tuning_t()
    _check(load().hist_batch_tune(b, arr, len(cols), _ptr(weights), int(n), ctypes.byref(r)), "hist_batch_tune")
    return {f: getattr(r, f) for f, _ in hist_batch_tuning_t._fields_}


def hist_batch_configure(b: int, strategy: int, smem_bytes: int, cost_cap_tenths: int = 30,
                         pace_tiles: int = -1, blocks_per_sm: int = 2, events_per_thread: int = 4) -> dict:
    r = hist_batch_tuning_t()
    _check(load().hist_batch_configure(b, int(strategy), int(smem_bytes), int(cost_cap_tenths), int(pace_tiles),
                                       int(blocks_per_sm), int(events_per_thread), ctypes.byref(r)),
           "hist_batch_configure")
    return {f: getattr(r, f) for f, _ in hist_batch_tuning_t._fields_}


LOCATOR_MODES = {0: "affine", 1: "bsearch", 2: "learned", 3: "bucket"}


def hist_locator_mode(h: int, axis: int = 0) -> str:
    m = load().hist_locator_mode(h, int(axis))
    if m < 0:
        raise HistError(m, "hist_locator_mode")
    return LOCATOR_MODES[m]


def hist_fill_columns(h: int, cols, defines, filters, weights, n: int, stream=None) -> None:
    """Fused Filter/Define fill: ``cols`` device float64 tensors, ``defines``
    [(op, a, b)] per axis, ``filters`` [(col, op, value)]."""
    arr = _col_array(cols)
    d = (hist_define_t * max(len(defines), 1))(*[hist_define_t(int(o), int(a), int(b)) for o, a, b in defines])
    f = (hist_filter_t * max(len(filters), 1))(*[hist_filter_t(int(c), int(o), float(v)) for c, o, v in filters])
    _check(load().hist_fill_columns(h, arr, len(cols), ctypes.byref(d), ctypes.byref(f), len(filters),
                                    _ptr(weights), int(n), _stream_ptr(stream)), "hist_fill_columns")


def hist_sumw2(h: int, nbins_total: int):
    import numpy as np
    out = np.zeros(nbins_total, dtype=np.float64)
    _check(load().hist_sumw2(h, out.ctypes.data), "hist_sumw2")
    return out


def hist_fill_host(h: int, values, weights, n: int, bulk: int = 0, stream=None) -> None:
    """Pipelined fill from host memory: ``values`` and ``weights`` are CPU
    tensors (pinned for asynchronous copies) or numpy arrays, float64,
    contiguous; the caller keeps them alive until the stream passes."""
    def host_ptr(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            assert not a.is_cuda and a.is_contiguous()
            return a.data_ptr()
        import numpy as np
        assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"] and a.dtype == np.float64
        return a.ctypes.data
    _check(load().hist_fill_host(h, host_ptr(values), host_ptr(weights), int(n), int(bulk), _stream_ptr(stream)),
           "hist_fill_host")


def hist_set_kernel_timing(h: int, on: bool) -> None:
    _check(load().hist_set_kernel_timing(h, int(bool(on))), "hist_set_kernel_timing")


def hist_kernel_time(h: int):
    """(summed fill-kernel milliseconds, timed launches) since the last call."""
    ms = ctypes.c_double()
    k = ctypes.c_int64()
    _check(load().hist_kernel_time(h, ctypes.byref(ms), ctypes.byref(k)), "hist_kernel_time")
    return ms.value, k.value


def hist_batch_free(b: int) -> None:
    load().hist_batch_free(b)


class Batch:
    """Owns a batch over Hist objects (which must outlive it)."""

    def __init__(self, hists, col_of_hist, flags: int = 0):
        self.hists = list(hists)
        self.b = hist_batch_create([h.h for h in self.hists], col_of_hist, flags)

    def fill(self, cols, weights=None, stream=None) -> None:
        n = int(cols[0].shape[-1])
        hist_batch_fill(self.b, list(cols), weights, n, stream)

    def tune(self, cols, weights=None) -> dict:
        return hist_batch_tune(self.b, list(cols), weights, int(cols[0].shape[-1]))

    def configure(self, strategy: int, smem_bytes: int, cost_cap_tenths: int = 30, pace_tiles: int = -1,
                  blocks_per_sm: int = 2, events_per_thread: int = 4) -> dict:
        return hist_batch_configure(self.b, strategy, smem_bytes, cost_cap_tenths, pace_tiles, blocks_per_sm,
                                    events_per_thread)

    def close(self) -> None:
        if self.b:
            hist_batch_free(self.b)
            self.b = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- owner ------

class Hist:
    """Owns one booked histogram.  ``values`` is a CUDA float64 tensor of
    shape (ndim, n) (or (n,) in 1D), ``weights`` a CUDA float64 tensor (n,)
    or None; fills run on the current torch stream and accumulate."""

    def __init__(self, axes, flags: int = 0):
        self.axes = axes
        self.ndim = len(axes)
        self.flags = flags
        self.h = hist_book(axes, flags)

    def fill(self, values, weights=None, stream=None) -> None:
        n = int(values.shape[-1])
        if values.dim() == 1:
            assert self.ndim == 1
        else:
            assert values.shape[0] == self.ndim and values.is_contiguous()
        if weights is not None:
            assert weights.shape == (n,) and weights.is_contiguous()
        hist_fill_bulk(self.h, values, weights, n, stream)

    def fill_columns(self, cols, defines, filters=(), weights=None, stream=None) -> None:
        hist_fill_columns(self.h, list(cols), list(defines), list(filters), weights, int(cols[0].shape[-1]), stream)

    def sumw2(self):
        return hist_sumw2(self.h, self.nbins_total)

    def fill_host(self, values, weights=None, bulk: int = 0, stream=None) -> None:
        n = int(values.shape[-1])
        hist_fill_host(self.h, values, weights, n, bulk, stream)

    def locate(self, values, out=None, stream=None):
        import torch
        n = int(values.shape[-1])
        if out is None:
            out = torch.empty(n, dtype=torch.int64, device=values.device)
        hist_locate(self.h, values, n, out, stream)
        return out

    def train_locator(self, axis: int = 0, **kw) -> dict:
        return hist_train_locator(self.h, axis, **kw)

    def result(self):
        return hist_result(self.h)

    def counts(self):
        return hist_counts(self.h)

    def reset(self):
        hist_reset(self.h)

    @property
    def nbins_total(self) -> int:
        return hist_nbins_total(self.h)

    def close(self) -> None:
        if self.h:
            hist_free(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
