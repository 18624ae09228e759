"""Full-size parity of the batched and learned-locator workloads.

The 64-histogram batch (5e7 weighted events on three columns, 10 .. 1e5 bins
per histogram, fixed and variable axes) and the 8 variable axes of 1e4 .. 1e6
mixture-quantile edges (1e8 unit-weight values) against the chunk-parallel
CPU oracle on all host cores, in every form the benchmark times: plain
per-histogram fills, the tuned batch, and each batch strategy pinned; for the
8-axis workload with the bucket-map, binary-search and learned locators.
Counts and unit-weight bins bit-exact; weighted bins and statistics within
1e-12 of the sum of |terms| (Sec. 3.1 of the paper defines the fill; the
oracle restates it).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import assert_sums_close, to_device

pytestmark = pytest.mark.gpu

RTOL = 1e-12
N4 = 50_000_000
N5 = 100_000_000


def _threads():
    return max(1, len(os.sched_getaffinity(0)))


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def cfg4_ref():
    bw = W.cfg4(n=N4)
    refs = [oracle.fill([ax], bw.columns[c].reshape(1, -1), bw.weights, threads=_threads())
            for ax, c in zip(bw.axes, bw.col_of_hist)]
    return bw, refs


# FP32 compensated bins (HIST_PREC_FP32C): the stated per-bin bound
# 2^-48 ((m + 1)^2 + 1) A + B 2^-53 A grows with m, the bin's entries in one
# block, which reach ~1e4 here (5e7 events over a few hundred blocks into 10
# bins); the errors measured at this size reach ~1.5e-12 A.  A compensation
# that lost the TwoSum error term would be near 2^-24 m-fold worse.
RTOL_FP32C_FULL = 1e-11


def _check_weighted(results, bw, refs, what, counts=None, rtol_bins=RTOL):
    for i, ((bins, stats), ref) in enumerate(zip(results, refs)):
        if counts is not None:
            assert np.array_equal(counts[i], ref.counts), f"{what} hist {i}: counts differ"
        assert_sums_close(bins, ref.bins_acc, ref.bins_abs, rtol_bins, f"{what} hist {i} bins")
        assert stats[0] == ref.stats_acc[0], f"{what} hist {i}: entries"
        assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"{what} hist {i} stats")


def test_cfg4_full_size_plain_and_batched(B, cfg4_ref):
    """64 histograms x 5e7 events: the 64 plain fills (with per-bin counts),
    the batch after tuning on a 4e6-event sample, and the wide, sliced and
    partitioned strategies pinned -- each against the oracle."""
    import torch
    bw, refs = cfg4_ref
    cols = [to_device(np.ascontiguousarray(bw.columns[c])) for c in range(3)]
    w = to_device(bw.weights)
    # plain: one launch per histogram
    hists = [B.Hist([ax], B.HIST_TRACK_COUNTS) for ax in bw.axes]
    try:
        for h, c in zip(hists, bw.col_of_hist):
            h.fill(cols[c], w)
        torch.cuda.synchronize()
        _check_weighted([h.result() for h in hists], bw, refs, "plain", counts=[h.counts() for h in hists])
    finally:
        for h in hists:
            h.close()
    # batched: tuned, then each strategy pinned; the FP32 compensated batch
    plans = [("tuned", None, 0), ("wide", (0, 48 << 10, 30, -1, 2, 2), 0),
             ("sliced", (1, 200 << 10, 30, -1, 2, 4), 0), ("partitioned", (2, 100 << 10, 30, -1, 2, 4), 0),
             ("fp32c tuned", None, B.HIST_PREC_FP32C),
             ("fp32c partitioned", (2, 48 << 10, 30, -1, 2, 4), B.HIST_PREC_FP32C)]
    for name, cfg, prec in plans:
        hists = [B.Hist([ax], prec) for ax in bw.axes]
        batch = None
        try:
            batch = B.Batch(hists, bw.col_of_hist, B.HIST_BATCH_GRAPH)
            if cfg is None:
                batch.tune([c[:4_000_000] for c in cols], w[:4_000_000])
            else:
                batch.configure(*cfg)
            batch.fill(cols, w)
            torch.cuda.synchronize()
            _check_weighted([h.result() for h in hists], bw, refs, f"batch {name}",
                            rtol_bins=RTOL_FP32C_FULL if prec else RTOL)
        finally:
            if batch is not None:
                batch.close()
            for h in hists:
                h.close()


@pytest.fixture(scope="module")
def cfg5_ref():
    bw = W.cfg5(n=N5)
    refs = [oracle.fill([ax], bw.columns, None, threads=_threads()) for ax in bw.axes]
    return bw, refs


def _check_unit(results, refs, what, counts=None):
    for i, ((bins, stats), ref) in enumerate(zip(results, refs)):
        if counts is not None:
            assert np.array_equal(counts[i], ref.counts), f"{what} hist {i}: counts differ"
        bad = np.flatnonzero(bins != ref.counts.astype(np.float64))
        assert bad.size == 0, f"{what} hist {i}: {bad.size} bins differ, first {bad[:5]}"
        assert stats[0] == ref.stats_acc[0]
        assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"{what} hist {i} stats")


@pytest.mark.parametrize("locator", ["default", "bsearch", "learned"])
def test_cfg5_full_size_locators(B, cfg5_ref, locator):
    """8 axes with 1e4 .. 1e6 mixture-quantile edges, 1e8 mixture values,
    unit weights: plain fills and the tuned batch, with the default
    (bucket-map) locator, plain binary search, and the trained learned
    locator -- bins bit-exact against the oracle."""
    import torch
    bw, refs = cfg5_ref
    col = to_device(np.ascontiguousarray(bw.columns[0]))
    flags = B.HIST_LOCATOR_BSEARCH if locator != "default" else 0
    hists = [B.Hist([ax], flags) for ax in bw.axes]
    batch = None
    try:
        modes = [B.hist_locator_mode(h.h, 0) for h in hists]
        if locator == "learned":
            reps = [h.train_locator(0) for h in hists]
            assert all(0 <= r["window"] <= 64 for r in reps)
            modes = [B.hist_locator_mode(h.h, 0) for h in hists]
            assert all(m == "learned" for m in modes), modes
        elif locator == "bsearch":
            assert all(m == "bsearch" for m in modes), modes
        for h in hists:
            h.fill(col, None)
        torch.cuda.synchronize()
        _check_unit([h.result() for h in hists], refs, f"plain {locator}", counts=[h.counts() for h in hists])
        for h in hists:
            h.reset()
        batch = B.Batch(hists, bw.col_of_hist, B.HIST_BATCH_GRAPH)
        rep = batch.tune([col[:8_000_000]], None)
        batch.fill([col], None)
        torch.cuda.synchronize()
        _check_unit([h.result() for h in hists], refs, f"batch {locator} (tuned strategy {rep['strategy']})")
        # the partitioned strategy pinned (events partitioned by range)
        for h in hists:
            h.reset()
        batch.configure(2, 100 << 10)
        batch.fill([col], None)
        torch.cuda.synchronize()
        _check_unit([h.result() for h in hists], refs, f"partitioned batch {locator}")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


def test_fill_beyond_2_31_events(B):
    """One plain fill of more than 2^31 events (an odd count): the fill's
    64-bit event indices, its per-thread pair counts and its odd last event
    past 2^31.  Unit weights on 100 fixed bins with flows; counts bit-exact
    against the chunk-parallel oracle, the entry count equal to n."""
    import torch
    phys = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    n = (1 << 31) + (1 << 20) + 3
    if phys < 8 * n * 3:
        pytest.skip("host memory too small for the oracle's copy of the column")
    g = torch.Generator(device="cuda")
    g.manual_seed(17)
    x = torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
    x.mul_(1.2).sub_(0.1)
    ax = W.fixed(100, 0.0, 1.0)
    h = B.Hist([ax])
    try:
        h.fill(x)
        bins, stats = h.result()
    finally:
        h.close()
    xh = x.cpu().numpy()
    del x
    torch.cuda.empty_cache()
    ref = oracle.fill([ax], xh.reshape(1, -1), threads=_threads())
    assert stats[0] == n
    assert np.array_equal(bins, ref.counts.astype(np.float64)), "counts differ beyond 2^31 events"
    assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, "stats beyond 2^31 events")
