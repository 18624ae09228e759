"""The bucket-map locator of variable axes (the default when an axis has a
usable map) against the oracle and against the plain binary search: the
same bins for every threshold and its neighbouring doubles, signed zeros,
infinities, NaN, subnormals and huge values, and the same counts from a
fill, on axes chosen to exercise both maps (linear, logarithmic), ranges
spanning zero, tiny and huge magnitudes, and an axis too bunched for any
map (which must fall back to the binary search)."""
import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import edge_probe_values, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


def _axes():
    rng = np.random.default_rng(41)
    bunched = np.concatenate([np.linspace(0.0, 1e-6, 2000), np.linspace(1.0, 100.0, 10)])
    return [
        ("log500", W.variable(W.log_edges(500, 0.0, 3.0)), "bucket"),
        ("jittered_phi", W.variable(W.jittered_edges(1000, -np.pi, np.pi, rng)), "bucket"),
        ("mixture1e4", W.variable(W.mixture_quantile_edges(10_000)), "bucket"),
        ("tiny_log", W.variable(W.log_edges(300, -30.0, -20.0)), "bucket"),
        ("spans_zero", W.variable([-3.0, -1.0, -0.0, 0.5, 10.0]), None),
        ("huge", W.variable([-1e300, -1.0, 0.0, 1e-300, 1.0, 1e300]), None),
        ("normal_sorted", W.variable(np.sort(rng.normal(0, 1, 20001))), None),
        ("bunched", W.variable(bunched), "bsearch"),
    ]


@pytest.mark.parametrize("name,axis,mode", _axes(), ids=[a[0] for a in _axes()])
def test_bucket_locate_bit_exact(B, name, axis, mode):
    import torch
    rng = np.random.default_rng(7)
    T = B.hist_axis_thresholds(axis)
    x = edge_probe_values(axis, T, rng, nrand=20_000)
    ref = oracle.locate([axis], x.reshape(1, -1))
    h = B.Hist([axis])
    hb = B.Hist([axis], B.HIST_LOCATOR_BSEARCH)
    try:
        got_mode = B.hist_locator_mode(h.h, 0)
        assert B.hist_locator_mode(hb.h, 0) == "bsearch"
        if mode is not None:
            assert got_mode == mode, f"{name}: locator {got_mode}, expected {mode}"
        got = h.locate(to_device(x.reshape(1, -1))).cpu().numpy()
        got_bs = hb.locate(to_device(x.reshape(1, -1))).cpu().numpy()
        torch.cuda.synchronize()
    finally:
        h.close()
        hb.close()
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, f"{name} ({got_mode}): {bad.size} mismatches, e.g. x={x[bad[:5]]!r} got {got[bad[:5]]} ref {ref[bad[:5]]}"
    assert np.array_equal(got_bs, ref)


@pytest.mark.parametrize("name,axis,mode", _axes()[:4], ids=[a[0] for a in _axes()[:4]])
def test_bucket_fill_counts_equal_binary_search(B, name, axis, mode):
    """A weighted fill through the shared-memory fill kernel: the bucket
    locator and the binary search give identical counts and bins."""
    rng = np.random.default_rng(9)
    edges = np.asarray(axis["edges"])
    lo, hi = edges[0], edges[-1]
    x = np.concatenate([rng.uniform(lo, hi, 400_000), edges, np.nextafter(edges, -np.inf)])
    w = rng.uniform(0.5, 1.5, x.shape[0])
    out = []
    for flags in (B.HIST_TRACK_COUNTS, B.HIST_TRACK_COUNTS | B.HIST_LOCATOR_BSEARCH):
        h = B.Hist([axis], flags)
        try:
            h.fill(to_device(x), to_device(w))
            bins, _ = h.result()
            out.append((h.counts(), bins))
        finally:
            h.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])  # exact fixed-point bins: order-independent
    ref = oracle.fill([axis], x.reshape(1, -1), w)
    assert np.array_equal(out[0][0], ref.counts)


@pytest.mark.parametrize("name,axis,mode", _axes(), ids=[a[0] for a in _axes()])
def test_bucket_unit_fill_counts_exact(B, name, axis, mode):
    """Unit weights through the fill kernels on every axis (bucket map, pair
    table, binary-search fallback): counts bit-exact against the oracle,
    including the edges, their predecessors and the special values."""
    import torch
    rng = np.random.default_rng(13)
    T = B.hist_axis_thresholds(axis)
    x = np.concatenate([edge_probe_values(axis, T, rng, nrand=200_000), np.zeros(5)])
    h = B.Hist([axis])
    try:
        h.fill(to_device(x.reshape(1, -1)), None)
        torch.cuda.synchronize()
        got = h.counts()
        bins, stats = h.result()
    finally:
        h.close()
    ref = oracle.fill([axis], x.reshape(1, -1), None)
    assert np.array_equal(got, ref.counts), f"{name}: counts differ at {np.flatnonzero(got != ref.counts)[:10]}"
    assert np.array_equal(bins, ref.counts.astype(np.float64))
    assert stats[0] == ref.stats_acc[0]
