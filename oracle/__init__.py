"""CPU oracle for bulk histogram filling (Python side).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  The product path (the CUDA
library under ``paper_2401_13310_gb300/`` and its binding) never imports it,
and the two share no code.

The arithmetic lives in ``hist_oracle.c`` (plain C, compiled with
``-ffp-contract=off``); this module builds it with gcc and marshals numpy
arrays through ctypes.  What it computes follows Sec. 3.1 and Sec. 3.2 of
Chen, Dessole and Varbanescu (2024): per event, find the bin (fixed-width
formula or binary search over edges, underflow bin 0, overflow bin nbins+1,
per axis then linearised), add the weight to the bin, and update the
statistics sums.  The readings taken where the paper is silent are listed at
the top of ``hist_oracle.c``.

Axes are plain dicts: ``{"kind": "fixed", "nbins": n, "xmin": a, "xmax": b}``
or ``{"kind": "variable", "edges": array_of_n_plus_1}``.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import math

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hist_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hist_oracle.c into liboracle.so next to it (gcc, no FMA)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


class _Axis(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nbins", ctypes.c_int32),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("edges", ctypes.c_void_p)]


_P = ctypes.c_void_p


def _configure(lib):
    lib.oracle_find_bin_fixed.restype = ctypes.c_int32
    lib.oracle_find_bin_fixed.argtypes = [ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double]
    lib.oracle_find_bin_variable.restype = ctypes.c_int32
    lib.oracle_find_bin_variable.argtypes = [ctypes.c_int32, _P, ctypes.c_double]
    lib.oracle_num_stats.restype = ctypes.c_int32
    lib.oracle_num_stats.argtypes = [ctypes.c_int32]
    lib.oracle_locate.restype = None
    lib.oracle_locate.argtypes = [_P, ctypes.c_int32, _P, ctypes.c_int64, _P]
    lib.oracle_locate_mt.restype = ctypes.c_int
    lib.oracle_locate_mt.argtypes = [_P, ctypes.c_int32, _P, ctypes.c_int64,
                                     ctypes.c_int32, _P]
    lib.oracle_fill.restype = ctypes.c_int
    lib.oracle_fill.argtypes = [_P, ctypes.c_int32, _P, _P, ctypes.c_int64,
                                ctypes.c_int32] + [_P] * 9
    lib.oracle_fill_mt.restype = ctypes.c_int
    lib.oracle_fill_mt.argtypes = [_P, ctypes.c_int32, _P, _P, ctypes.c_int64,
                                   ctypes.c_int32, ctypes.c_int32] + [_P] * 9
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Run the oracle API against another build of hist_oracle.c (the pin
    tests use this to check that planted mistakes are caught)."""
    global _lib
    lib = _configure(ctypes.CDLL(path))
    with _lock:
        saved = _lib
        _lib = lib
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a (test-modified) copy of the oracle source with the same flags."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", *_CFLAGS, "-o", out_path, c_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _axes_struct(axes):
    """Build the C axis array; returns (array, keepalive list)."""
    arr = (_Axis * len(axes))()
    keep = []
    for d, ax in enumerate(axes):
        if ax["kind"] == "fixed":
            arr[d].kind = 0
            arr[d].nbins = int(ax["nbins"])
            arr[d].xmin = float(ax["xmin"])
            arr[d].xmax = float(ax["xmax"])
            arr[d].edges = None
        elif ax["kind"] == "variable":
            e = np.ascontiguousarray(ax["edges"], dtype=np.float64)
            keep.append(e)
            arr[d].kind = 1
            arr[d].nbins = int(e.shape[0] - 1)
            arr[d].edges = e.ctypes.data
        else:
            raise ValueError(f"unknown axis kind {ax['kind']!r}")
    return arr, keep


def nbins_total(axes) -> int:
    nb = 1
    for ax in axes:
        n = int(ax["nbins"]) if ax["kind"] == "fixed" else len(ax["edges"]) - 1
        nb *= n + 2
    return nb


def num_stats(ndim: int) -> int:
    return {1: 5, 2: 8, 3: 12}[ndim]


def find_bin_fixed(nbins: int, xmin: float, xmax: float, x: float) -> int:
    """Sec. 3.1 fixed-width find-bin of one coordinate (readings R2-R4)."""
    return int(_load().oracle_find_bin_fixed(nbins, xmin, xmax, x))


def find_bin_variable(edges, x: float) -> int:
    """Sec. 3.1 variable-width find-bin of one coordinate (reading R1)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    return int(_load().oracle_find_bin_variable(e.shape[0] - 1, e.ctypes.data, x))


def _values2d(values, ndim):
    v = np.ascontiguousarray(values, dtype=np.float64)
    if v.ndim == 1:
        v = v.reshape(1, -1)
    if v.shape[0] != ndim:
        raise ValueError("values must have shape (ndim, n)")
    return v


def locate(axes, values, threads: int = 1) -> np.ndarray:
    """Linear bin index of every event (find-bin per axis, x fastest)."""
    lib = _load()
    arr, keep = _axes_struct(axes)
    v = _values2d(values, len(axes))
    n = v.shape[1]
    out = np.empty(n, dtype=np.int64)
    if threads <= 1:
        lib.oracle_locate(ctypes.addressof(arr), len(axes), _ptr(v), n, _ptr(out))
    else:
        rc = lib.oracle_locate_mt(ctypes.addressof(arr), len(axes), _ptr(v), n,
                                  threads, _ptr(out))
        if rc != 0:
            raise RuntimeError(f"oracle_locate_mt failed ({rc})")
    del keep
    return out


@dataclass
class FillResult:
    counts: np.ndarray      # uint64 [nbins_total]: entries per bin
    bins_seq: np.ndarray    # float64: event-order binary64 sum of weights
    bins_acc: np.ndarray    # float64: compensated sum of weights (reference)
    bins_abs: np.ndarray    # float64: sum of |w| per bin (tolerance scale)
    stats_seq: np.ndarray   # float64 [ns]: [N, sum w, sum w^2, sum wx, sum wx^2, ...]
    stats_acc: np.ndarray
    stats_abs: np.ndarray


class Accumulator:
    """Running oracle histogram: repeated fill() calls accumulate (a fill
    adds to the previous state and never overwrites it)."""

    def __init__(self, axes, stat_overflows: bool = False):
        self.axes = axes
        self.stat_overflows = bool(stat_overflows)
        nb = nbins_total(axes)
        ns = num_stats(len(axes))
        self.counts = np.zeros(nb, dtype=np.uint64)
        self.bins_seq = np.zeros(nb)
        self.bins_acc_s = np.zeros(nb)
        self.bins_acc_c = np.zeros(nb)
        self.bins_abs = np.zeros(nb)
        self.stats_seq = np.zeros(ns)
        self.stats_acc_s = np.zeros(ns)
        self.stats_acc_c = np.zeros(ns)
        self.stats_abs = np.zeros(ns)

    def fill(self, values, weights=None, threads: int = 1) -> None:
        lib = _load()
        arr, keep = _axes_struct(self.axes)
        v = _values2d(values, len(self.axes))
        n = v.shape[1]
        w = None
        if weights is not None:
            w = np.ascontiguousarray(weights, dtype=np.float64)
            if w.shape != (n,):
                raise ValueError("weights must have shape (n,)")
        outs = [self.counts, self.bins_seq, self.bins_acc_s, self.bins_acc_c,
                self.bins_abs, self.stats_seq, self.stats_acc_s, self.stats_acc_c,
                self.stats_abs]
        if threads <= 1:
            rc = lib.oracle_fill(ctypes.addressof(arr), len(self.axes), _ptr(v), _ptr(w),
                                 n, int(self.stat_overflows), *[_ptr(o) for o in outs])
        else:
            rc = lib.oracle_fill_mt(ctypes.addressof(arr), len(self.axes), _ptr(v),
                                    _ptr(w), n, int(self.stat_overflows), int(threads),
                                    *[_ptr(o) for o in outs])
        del keep
        if rc != 0:
            raise RuntimeError(f"oracle fill failed ({rc})")

    def result(self) -> FillResult:
        return FillResult(self.counts.copy(), self.bins_seq.copy(),
                          self.bins_acc_s + self.bins_acc_c, self.bins_abs.copy(),
                          self.stats_seq.copy(), self.stats_acc_s + self.stats_acc_c,
                          self.stats_abs.copy())


def fill(axes, values, weights=None, stat_overflows: bool = False,
         threads: int = 1) -> FillResult:
    """One bulk fill of a fresh histogram (Sec. 3.1 steps 1-3 per event)."""
    acc = Accumulator(axes, stat_overflows)
    acc.fill(values, weights, threads=threads)
    return acc.result()


def exact_stats(axes, values, weights=None, stat_overflows: bool = False):
    """The statistics as the exact sums of their rounded terms, each sum
    rounded once (math.fsum is the correctly rounded sum of its inputs),
    over the in-range entries (R5: every axis in range).  The terms are
    those of R6, binary64, each product rounded left to right: 1D w, w*w,
    w*x, (w*x)*x; 2D adds w*y, (w*y)*y, (w*x)*y; 3D adds w*z, (w*z)*z,
    (w*x)*z, (w*y)*z.  Returns [sum w, sum w^2, sum wx, ...] (4, 7 or 11
    values); NaN when a term is NaN or infinities of both signs meet, +-inf
    for infinities of one sign."""
    ndim = len(axes)
    v = np.asarray(values, dtype=np.float64).reshape(ndim, -1)
    n = v.shape[1]
    w = np.ones(n) if weights is None else np.asarray(weights, dtype=np.float64)
    m = np.ones(n, dtype=bool)
    if not stat_overflows:
        for d, ax in enumerate(axes):
            b = locate([ax], v[d].reshape(1, -1))
            nb = nbins_total([ax])
            m &= (b >= 1) & (b <= nb - 2)
    v, w = v[:, m], w[m]
    with np.errstate(all="ignore"):
        x = v[0]
        wx = w * x
        terms = [w, w * w, wx, wx * x]
        if ndim >= 2:
            y = v[1]
            wy = w * y
            terms += [wy, wy * y, wx * y]
        if ndim >= 3:
            z = v[2]
            wz = w * z
            terms += [wz, wz * z, wx * z, wy * z]
    out = []
    for t in terms:
        if np.isnan(t).any() or (np.isposinf(t).any() and np.isneginf(t).any()):
            out.append(math.nan)
        elif np.isposinf(t).any():
            out.append(math.inf)
        elif np.isneginf(t).any():
            out.append(-math.inf)
        else:
            out.append(math.fsum(t.tolist()))
    return out


# Filter/Define operation codes (the library's HIST_DEF_* / HIST_FLT_*).
DEF_COL, DEF_SUMSQ, DEF_HYPOT, DEF_MUL, DEF_ADD, DEF_SUB = range(6)
FLT_NE, FLT_EQ, FLT_LT, FLT_LE, FLT_GT, FLT_GE = range(6)


def define_filter(columns, defines, filters):
    """The paper's RDataFrame example (Sec. 2, Listing 1) restated: rows
    pass when every filter (column <op> constant, binary64 comparison)
    holds; each axis coordinate is its define evaluated in binary64, one
    rounding per operation, left to right (a*a + b*b is fl(fl(a*a) +
    fl(b*b)); sqrt correctly rounded).  Returns (mask, values[ndim][n])."""
    cols = [np.asarray(c, dtype=np.float64) for c in columns]
    n = cols[0].shape[0]
    mask = np.ones(n, dtype=bool)
    with np.errstate(invalid="ignore"):
        for c, op, v in filters:
            a = cols[c]
            mask &= {FLT_NE: a != v, FLT_EQ: a == v, FLT_LT: a < v, FLT_LE: a <= v,
                     FLT_GT: a > v, FLT_GE: a >= v}[op]
    vals = []
    with np.errstate(all="ignore"):
        for op, a, b in defines:
            x, y = cols[a], cols[b]
            if op == DEF_COL:
                vals.append(x.copy())
            elif op == DEF_SUMSQ:
                vals.append(x * x + y * y)
            elif op == DEF_HYPOT:
                vals.append(np.sqrt(x * x + y * y))
            elif op == DEF_MUL:
                vals.append(x * y)
            elif op == DEF_ADD:
                vals.append(x + y)
            else:
                vals.append(x - y)
    return mask, np.stack(vals)


def sumw2(axes, values, weights=None, threads: int = 1):
    """Per-bin sum of squared weights (ROOT's Sumw2, the input of the bin
    errors; the paper's statistics sums stop at the per-histogram level):
    each entry adds its rounded w*w to its bin -- the per-bin weighted sum
    of this oracle with the squared weights as weights; unit weights give
    the entry counts.  Returns (compensated sums, sums of |w*w|)."""
    if weights is None:
        r = fill(axes, values, None, threads=threads)
        c = r.counts.astype(np.float64)
        return c, c.copy()
    w = np.ascontiguousarray(weights, dtype=np.float64)
    r = fill(axes, values, w * w, threads=threads)
    return r.bins_acc, r.bins_abs
