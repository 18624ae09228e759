"""The allocation-free fill (hist_fill_bulk_noalloc) against the regular
entry points (hist_book + hist_fill_bulk + hist_result), through the C ABI.

hist_fill_bulk_noalloc exists for callers that cannot call cudaMalloc (code
under another framework's memory manager, allocation-free real-time loops):
its scratch is one fixed library array shared by all calls.  Two calls in a
row must each give the same answer as the regular path on the same bulk --
the second call must not see the first call's leftovers.  This file sorts
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import assert_sums_close, gpu_fill, to_device

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # the tolerance of the parity tests, relative to sum |term|


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


def _noalloc(B, axis, x, w, flags=0):
    import torch
    nb = (axis["nbins"] if axis["kind"] == "fixed" else len(axis["edges"]) - 1) + 2
    bins = torch.full((nb,), float("nan"), dtype=torch.float64, device="cuda")
    stats = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    xd = to_device(x)
    wd = to_device(w)
    B.hist_fill_bulk_noalloc(axis, xd, wd, x.shape[0], flags, bins, stats)
    torch.cuda.synchronize()
    return bins.cpu().numpy(), stats.cpu().numpy()


def _compare(B, axis, x, w, flags=0, what=""):
    got_bins, got_stats = _noalloc(B, axis, x, w, flags)
    ref_bins, ref_stats, _ = gpu_fill([axis], x.reshape(1, -1), w, flags=flags)
    scale = oracle.fill([axis], x.reshape(1, -1), w, stat_overflows=bool(flags & B.HIST_STAT_OVERFLOWS))
    assert_sums_close(got_bins, ref_bins, scale.bins_abs, RTOL, f"{what} bins")
    assert got_stats[0] == ref_stats[0]
    assert_sums_close(got_stats[1:], ref_stats[1:], scale.stats_abs[1:], RTOL, f"{what} stats")


def test_noalloc_matches_regular_path_twice_in_a_row(B):
    rng = np.random.default_rng(21)
    axis = W.fixed(1000, -5.0, 5.0)
    for call in range(2):
        n = 300_001 + 7 * call
        x = rng.normal(0, 1.5, n)
        w = rng.uniform(0.5, 1.5, n)
        _compare(B, axis, x, w, what=f"weighted call {call}")


def test_noalloc_unit_and_variable_axis_twice_in_a_row(B):
    rng = np.random.default_rng(22)
    axis = W.variable(W.log_edges(500, 0.0, 3.0))
    for call in range(2):
        x = rng.exponential(30.0, 200_003 + call)
        _compare(B, axis, x, None, what=f"unit call {call}")
    # a smaller axis after a larger one, with flows in the statistics
    axis2 = W.fixed(10, 0.0, 1.0)
    x = rng.uniform(-0.5, 1.5, 50_001)
    w = rng.uniform(0.5, 1.5, 50_001)
    _compare(B, axis2, x, w, flags=B.HIST_STAT_OVERFLOWS, what="small axis")


def test_noalloc_rejects_oversized_axis(B):
    import torch
    axis = W.fixed(1023, 0.0, 1.0)  # 1025 bins with flows: one above the maximum
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1025, dtype=torch.float64, device="cuda")
    st = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(B.HistError) as e:
        B.hist_fill_bulk_noalloc(axis, x, None, 8, 0, out, st)
    assert e.value.code == B.HIST_ERR_TOO_LARGE
