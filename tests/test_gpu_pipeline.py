"""The pipelined host-memory fill (hist_fill_host): bulks copied into two
device slots on the histogram's copy stream while the previous bulk fills.
Same events, same results as hist_fill_bulk from device memory (the exact
fixed-point bins bit-identical whatever the bulk size), for pinned torch
tensors and pageable numpy arrays, ragged bulk sizes (including the paper's
32768-event bulks) and 1D and 2D histograms."""
import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import assert_sums_close, gpu_fill

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


def _host_fill(B, axes, values, weights, bulk, pinned, flags=0):
    import torch
    v = np.ascontiguousarray(values)
    w = None if weights is None else np.ascontiguousarray(weights)
    if pinned:
        v = torch.from_numpy(v).pin_memory()
        w = None if w is None else torch.from_numpy(w).pin_memory()
    h = B.Hist(axes, flags)
    try:
        h.fill_host(v, w, bulk=bulk)
        torch.cuda.synchronize()
        bins, stats = h.result()
        counts = h.counts() if (weights is None or flags & B.HIST_TRACK_COUNTS) else None
        return bins, stats, counts
    finally:
        h.close()


@pytest.mark.parametrize("name,n,bulk,pinned", [
    ("2a", 1_000_003, 32768, True), ("2b", 1_000_003, 65536, False), ("2a", 300_001, 0, True),
    ("1", 1 << 20, 100_000, True), ("3a", 500_001, 131_071, True), ("2b", 77, 1 << 20, True)])
def test_fill_host_matches_device_fill(B, name, n, bulk, pinned):
    wl = W.CONFIGS[name](n=n)
    flags = B.HIST_TRACK_COUNTS
    got = _host_fill(B, wl.axes, wl.values, wl.weights, bulk, pinned, flags)
    dev = gpu_fill(wl.axes, wl.values, wl.weights, flags=flags)
    assert np.array_equal(got[0], dev[0]), "bins differ from the device fill"
    assert np.array_equal(got[2], dev[2])
    ref = oracle.fill(wl.axes, wl.values, wl.weights)
    assert np.array_equal(got[2], ref.counts)
    assert got[1][0] == ref.stats_acc[0]
    assert_sums_close(got[1][1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"cfg{name} host stats")


def test_fill_host_accumulates_with_device_fills(B):
    import torch
    wl = W.cfg2a(n=400_000)
    h = B.Hist(wl.axes, B.HIST_TRACK_COUNTS)
    try:
        vd = torch.from_numpy(np.ascontiguousarray(wl.values[:, :200_000])).cuda()
        wd = torch.from_numpy(np.ascontiguousarray(wl.weights[:200_000])).cuda()
        h.fill(vd, wd)
        vh = torch.from_numpy(np.ascontiguousarray(wl.values[:, 200_000:])).pin_memory()
        wh = torch.from_numpy(np.ascontiguousarray(wl.weights[200_000:])).pin_memory()
        h.fill_host(vh, wh, bulk=50_000)
        h.fill_host(vh, wh, bulk=70_001)  # slots reused across calls
        torch.cuda.synchronize()
        bins, stats = h.result()
        counts = h.counts()
    finally:
        h.close()
    allv = np.concatenate([wl.values, wl.values[:, 200_000:]], axis=1)
    allw = np.concatenate([wl.weights, wl.weights[200_000:]])
    ref = oracle.fill(wl.axes, allv, allw)
    assert np.array_equal(counts, ref.counts)
    assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, "bins")
    assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, "stats")


def test_fill_host_graph_replays_and_recaptures(B):
    """Small bulks replay the whole pipelined fill as one CUDA graph: three
    calls with the same buffers accumulate like three fills; new buffers
    are captured anew."""
    import torch
    wl = W.cfg2b(n=250_001)
    v = torch.from_numpy(np.ascontiguousarray(wl.values)).pin_memory()
    w = torch.from_numpy(np.ascontiguousarray(wl.weights)).pin_memory()
    v2 = torch.from_numpy(np.ascontiguousarray(wl.values[:, :100_000])).pin_memory()
    w2 = torch.from_numpy(np.ascontiguousarray(wl.weights[:100_000])).pin_memory()
    h = B.Hist(wl.axes, B.HIST_TRACK_COUNTS)
    try:
        for _ in range(3):
            h.fill_host(v, w, bulk=32768)
        h.fill_host(v2, w2, bulk=32768)
        torch.cuda.synchronize()
        bins, stats = h.result()
        counts = h.counts()
    finally:
        h.close()
    allv = np.concatenate([wl.values] * 3 + [wl.values[:, :100_000]], axis=1)
    allw = np.concatenate([wl.weights] * 3 + [wl.weights[:100_000]])
    ref = oracle.fill(wl.axes, allv, allw)
    assert np.array_equal(counts, ref.counts)
    assert stats[0] == ref.stats_acc[0]
    assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, "bins")
    assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, "stats")


def test_fill_host_graph_survives_scratch_growth(B):
    """A replayed small-bulk graph holds the fill scratch; a larger device
    fill in between grows that scratch, and the next host fill must be
    captured anew (same results as plain fills)."""
    import torch
    wl = W.cfg2a(n=300_000)
    v = torch.from_numpy(np.ascontiguousarray(wl.values[:, :100_000])).pin_memory()
    w = torch.from_numpy(np.ascontiguousarray(wl.weights[:100_000])).pin_memory()
    big_v = torch.from_numpy(np.ascontiguousarray(wl.values)).cuda()
    big_w = torch.from_numpy(np.ascontiguousarray(wl.weights)).cuda()
    h = B.Hist(wl.axes, B.HIST_TRACK_COUNTS)
    try:
        h.fill_host(v, w, bulk=32768)  # captured with small-launch scratch
        h.fill(big_v, big_w)           # grows the scratch
        h.fill_host(v, w, bulk=32768)  # same arguments: replay must not use the old scratch
        torch.cuda.synchronize()
        bins, stats = h.result()
        counts = h.counts()
    finally:
        h.close()
    allv = np.concatenate([wl.values[:, :100_000], wl.values, wl.values[:, :100_000]], axis=1)
    allw = np.concatenate([wl.weights[:100_000], wl.weights, wl.weights[:100_000]])
    ref = oracle.fill(wl.axes, allv, allw)
    assert np.array_equal(counts, ref.counts)
    assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, "bins")
    assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, "stats")
