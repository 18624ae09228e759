"""The allocation-free fill (hist_fill_bulk_noalloc) against the CPU oracle
and against the regular entry points (hist_book + hist_fill_bulk +
hist_result), through the C ABI.

hist_fill_bulk_noalloc exists for callers that cannot call cudaMalloc (code
under another framework's memory manager, allocation-free real-time loops):
its scratch is one fixed library array shared by all calls.  Every call must
give the oracle's answer on its own bulk -- unit-weight bins and the entry
count bit-exact, weighted bins and statistics within 1e-12 of the sum of
|terms| -- and the same answer as the regular path; calls in a row must not
see the earlier calls' leftovers, whatever their sizes.  This file sorts last
so that a run stopping at the first failure has run everything else.
"""
import math

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
    ref = oracle.fill([axis], x.reshape(1, -1), w, stat_overflows=bool(flags & B.HIST_STAT_OVERFLOWS))
    # against the oracle
    if w is None:
        assert np.array_equal(got_bins, ref.counts.astype(np.float64)), f"{what}: unit-weight bins"
    else:
        assert_sums_close(got_bins, ref.bins_acc, ref.bins_abs, RTOL, f"{what} bins")
    assert got_stats[0] == ref.stats_acc[0] == x.shape[0], f"{what}: entries"
    assert_sums_close(got_stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"{what} stats")
    # against the regular path on the same bulk
    reg_bins, reg_stats, _ = gpu_fill([axis], x.reshape(1, -1), w, flags=flags)
    assert_sums_close(got_bins, reg_bins, ref.bins_abs, RTOL, f"{what} bins vs regular path")
    assert_sums_close(got_stats[1:], reg_stats[1:], ref.stats_abs[1:], RTOL, f"{what} stats vs regular path")


def test_noalloc_matches_oracle_twice_in_a_row(B):
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


def test_noalloc_largest_axes_then_a_small_one(B):
    """The largest accepted axes (nbins = 1022: 1024 bins with the flows,
    every threshold and per-block bin slot of the scratch in use), fixed and
    variable, unit and weighted, then a 5-bin axis that must not see their
    leftovers."""
    rng = np.random.default_rng(23)
    big_fixed = W.fixed(1022, -3.0, 3.0)
    big_var = W.variable(np.sort(rng.uniform(-3.0, 3.0, 1023)))
    n = 400_003
    x = rng.normal(0, 1.2, n)
    w = rng.uniform(0.5, 1.5, n)
    _compare(B, big_fixed, x, w, what="1022 fixed weighted")
    _compare(B, big_var, x, None, what="1022 variable unit")
    _compare(B, big_var, x, w, what="1022 variable weighted")
    small = W.fixed(5, -1.0, 1.0)
    xs = rng.uniform(-1.5, 1.5, 10_007)
    _compare(B, small, xs, None, what="5 bins after 1022")
    _compare(B, small, xs, rng.uniform(0.5, 1.5, 10_007), what="5 bins weighted after 1022")


def test_noalloc_odd_weights(B):
    """Weights outside the fixed-point window (zero, tiny, large), negative
    ones, and one +inf and one NaN weight in separate bins: the binary64
    words and their compensated sum, as the regular path forms them."""
    rng = np.random.default_rng(24)
    axis = W.fixed(40, -2.0, 2.0)
    n = 100_001
    x = rng.normal(0, 0.8, n)
    w = rng.uniform(-1.5, 1.5, n)
    w[::5] = 0.0
    w[1::7] = 1e3
    w[2::11] = -1e-4
    w[3::13] = 3e-9
    _compare(B, axis, x, w, what="odd weights")
    x2 = x.copy()
    w2 = w.copy()
    x2[:2] = [-1.99, 1.99]  # bins 1 and 40
    w2[:2] = [math.inf, math.nan]
    got_bins, got_stats = _noalloc(B, axis, x2, w2)
    reg_bins, reg_stats, _ = gpu_fill([axis], x2.reshape(1, -1), w2)
    ref = oracle.fill([axis], x2.reshape(1, -1), w2)
    assert got_bins[1] == math.inf and math.isnan(got_bins[40])
    assert_sums_close(got_bins, ref.bins_acc, ref.bins_abs, RTOL, "specials bins vs oracle")
    assert_sums_close(got_bins, reg_bins, ref.bins_abs, RTOL, "specials bins vs regular path")
    assert got_stats[0] == n and math.isnan(got_stats[1]) and math.isnan(reg_stats[1])


def test_noalloc_captured_in_a_cuda_graph_and_replayed(B):
    """After the first call on the device (its one-time set-up), the call is
    captured into a CUDA graph; every replay, with new events written into
    the same input buffers, gives the oracle's answer on those events.  The
    graph holds the whole call -- the thresholds as a kernel argument, the
    clearing of the scratch, the fill, the reduce and the finish -- and no
    copy from host memory."""
    import torch
    rng = np.random.default_rng(25)
    cases = ((W.variable(W.log_edges(500, 0.0, 3.0)), True), (W.fixed(1000, -5.0, 5.0), False))
    for axis, weighted in cases:
        n = 250_007
        nb = (axis["nbins"] if axis["kind"] == "fixed" else len(axis["edges"]) - 1) + 2
        xd = torch.zeros(n, dtype=torch.float64, device="cuda")
        wd = torch.ones(n, dtype=torch.float64, device="cuda") if weighted else None
        bins = torch.zeros(nb, dtype=torch.float64, device="cuda")
        stats = torch.zeros(5, dtype=torch.float64, device="cuda")
        B.hist_fill_bulk_noalloc(axis, xd, wd, n, 0, bins, stats)  # outside any capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            B.hist_fill_bulk_noalloc(axis, xd, wd, n, 0, bins, stats)
        for rep in range(3):
            what = f"{axis['kind']} replay {rep}"
            x = rng.exponential(30.0, n) if axis["kind"] == "variable" else rng.normal(0, 1.5, n)
            w = rng.uniform(-0.5, 1.5, n) if weighted else None
            xd.copy_(torch.from_numpy(x))
            if weighted:
                wd.copy_(torch.from_numpy(w))
            bins.fill_(float("nan"))
            stats.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            got_bins, got_stats = bins.cpu().numpy(), stats.cpu().numpy()
            ref = oracle.fill([axis], x.reshape(1, -1), w)
            if w is None:
                assert np.array_equal(got_bins, ref.counts.astype(np.float64)), f"{what}: unit-weight bins"
            else:
                assert_sums_close(got_bins, ref.bins_acc, ref.bins_abs, RTOL, f"{what} bins")
            assert got_stats[0] == n, f"{what}: entries"
            assert_sums_close(got_stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"{what} stats")
        del g


def test_noalloc_rejects_oversized_axis(B):
    import torch
    axis = W.fixed(1023, 0.0, 1.0)  # 1025 bins with flows: one above the maximum
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1025, dtype=torch.float64, device="cuda")
    st = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(B.HistError) as e:
        B.hist_fill_bulk_noalloc(axis, x, None, 8, 0, out, st)
    assert e.value.code == B.HIST_ERR_TOO_LARGE
