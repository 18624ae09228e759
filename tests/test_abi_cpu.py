"""CPU-only checks of the C ABI: the library builds for sm_103a, loads,
exports every function that include/hist.h declares, rejects bad arguments
on the host, and its host-side axis compiler produces exactly the thresholds
that the oracle's find-bin implies (no GPU needed for any of this)."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import _build
from paper_2401_13310_gb300 import binding as B
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import double_of_key

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return B.load()


def declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(hist_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "hist_book" in names and "hist_fill_bulk" in names and "hist_result" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_strerror_and_version(lib):
    assert lib.hist_version().decode().startswith("gb300-hist")
    assert B.strerror(B.HIST_ERR_AXIS) == "invalid axis"
    assert B.strerror(12345) == "unknown status"


@pytest.mark.parametrize("axis", [
    {"kind": "fixed", "nbins": 0, "xmin": 0.0, "xmax": 1.0},
    {"kind": "fixed", "nbins": 10, "xmin": 1.0, "xmax": 1.0},
    {"kind": "fixed", "nbins": 10, "xmin": 2.0, "xmax": 1.0},
    {"kind": "fixed", "nbins": 10, "xmin": math.nan, "xmax": 1.0},
    {"kind": "fixed", "nbins": 10, "xmin": -math.inf, "xmax": 1.0},
    {"kind": "fixed", "nbins": 10, "xmin": -1e308, "xmax": 1e308},
    {"kind": "variable", "edges": [0.0, 1.0, 1.0, 2.0]},
    {"kind": "variable", "edges": [0.0, 2.0, 1.0]},
    {"kind": "variable", "edges": [0.0, math.nan, 1.0]},
    {"kind": "variable", "edges": [0.0, math.inf]},
])
def test_invalid_axes_rejected_on_host(lib, axis):
    # Axis validation runs before any CUDA call, so this needs no GPU.
    with pytest.raises(B.HistError) as e:
        B.hist_book([axis])
    assert e.value.code == B.HIST_ERR_AXIS
    arr, keep = B.make_axes([axis])
    out = np.zeros(8, dtype=np.int64)
    if axis.get("nbins", 1) >= 1 and arr[0].nbins >= 1:
        out = np.zeros(int(arr[0].nbins) + 3, dtype=np.int64)
        assert lib.hist_axis_thresholds(arr, out.ctypes.data) == B.HIST_ERR_AXIS


def test_host_argument_errors(lib):
    assert lib.hist_fill_bulk(None, None, None, 10, None) == B.HIST_ERR_ARG
    assert lib.hist_result(None, None, None) == B.HIST_ERR_ARG
    assert lib.hist_counts(None, None) == B.HIST_ERR_ARG
    assert lib.hist_reset(None) == B.HIST_ERR_ARG
    assert lib.hist_locate(None, None, 5, None, None) == B.HIST_ERR_ARG
    assert lib.hist_fill_host(None, None, None, 10, 0, None) == B.HIST_ERR_ARG
    assert lib.hist_fill_columns(None, None, 1, None, None, 0, None, 10, None) == B.HIST_ERR_ARG
    assert lib.hist_sumw2(None, None) == B.HIST_ERR_ARG
    assert lib.hist_locator_mode(None, 0) == B.HIST_ERR_ARG
    assert lib.hist_set_kernel_timing(None, 1) == B.HIST_ERR_ARG
    assert lib.hist_kernel_time(None, None, None) == B.HIST_ERR_ARG
    assert lib.hist_batch_fill(None, None, 0, None, 10, None) == B.HIST_ERR_ARG
    assert lib.hist_batch_tune(None, None, 0, None, 10, None) == B.HIST_ERR_ARG
    assert lib.hist_batch_configure(None, 0, 1 << 16, 30, -1, 2, 4, None) == B.HIST_ERR_ARG
    assert lib.hist_batch_create(None, 0, None, 0, None) == B.HIST_ERR_ARG
    assert lib.hist_train_locator(None, 0, None, None) == B.HIST_ERR_ARG
    lib.hist_batch_free(None)
    lib.hist_free(None)
    for bad in (1 << 20, 3 << 8):  # an unknown flag; an unknown locator
        with pytest.raises(B.HistError) as e:
            B.hist_book([{"kind": "fixed", "nbins": 1, "xmin": 0.0, "xmax": 1.0}], flags=bad)
        assert e.value.code == B.HIST_ERR_ARG
    with pytest.raises(B.HistError) as e:
        B.hist_book([{"kind": "fixed", "nbins": 1, "xmin": 0.0, "xmax": 1.0}], flags=1 << 20)
    assert e.value.code == B.HIST_ERR_ARG


def _check_thresholds(axis, T):
    """T[k] is the least key whose oracle bin is >= k (k = 1..nbins+1)."""
    if axis["kind"] == "fixed":
        nb = axis["nbins"]
        f = lambda x: oracle.find_bin_fixed(nb, axis["xmin"], axis["xmax"], x)  # noqa: E731
    else:
        e = np.asarray(axis["edges"])
        nb = len(e) - 1
        f = lambda x: oracle.find_bin_variable(e, x)  # noqa: E731
    assert T[0] == -(1 << 63) and T[nb + 2] == (1 << 63) - 1
    assert all(int(a) <= int(b) for a, b in zip(T, T[1:]))
    for k in range(1, nb + 2):
        t = int(T[k])
        assert f(double_of_key(t)) >= k, (k, t)
        if t - 1 >= -0x7FF0000000000000:
            assert f(double_of_key(t - 1)) < k, (k, t)


@pytest.mark.parametrize("axis", [
    W.fixed(100, 0.0, 1.0), W.fixed(1000, -5.0, 5.0), W.fixed(222, -1.0, 1.5),
    W.fixed(7, -0.3, 0.4), W.fixed(1, 2.0, 3.0), W.fixed(100, 0.0, 300.0),
    W.fixed(3163, -math.pi, math.pi), W.fixed(64, -1e-300, 1e-300), W.fixed(50, 1e15, 1e15 + 1.0),
    W.variable(W.log_edges(500, 0.0, 3.0)), W.variable([-3.0, -1.0, -0.0, 0.5, 10.0]),
])
def test_host_thresholds_match_oracle(lib, axis):
    T = B.hist_axis_thresholds(axis)
    _check_thresholds(axis, T)


def test_host_thresholds_random_fixed_axes(lib):
    rng = np.random.default_rng(11)
    for _ in range(40):
        nb = int(rng.integers(1, 400))
        xmin = float(rng.uniform(-100, 100))
        xmax = xmin + float(rng.choice([1e-6, 0.37, 1.0, 12.5, 1e4]))
        axis = W.fixed(nb, xmin, xmax)
        _check_thresholds(axis, B.hist_axis_thresholds(axis))


def test_no_host_fallback_without_a_gpu(lib):
    """The library has no CPU path: without a GPU, booking a valid
    histogram fails with HIST_ERR_CUDA instead of succeeding on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(B.HistError) as e:
        B.hist_book([{"kind": "fixed", "nbins": 10, "xmin": 0.0, "xmax": 1.0}])
    assert e.value.code == B.HIST_ERR_CUDA


def test_binding_fails_loudly_when_the_library_is_missing(tmp_path):
    """Loading a library that is not there raises; the binding has no
    fallback to fill with."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("from paper_2401_13310_gb300 import binding as B\n"
            "try:\n"
            f"    B.load({str(tmp_path / 'libhist.so')!r})\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "raised:" in r.stdout and "missing" in r.stdout
