"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Bin indices and counts must match bit for bit; weighted
bin contents and statistics must agree with the oracle's compensated sums to
1e-12 of the sum of |terms| (HIST_PREC_FP64 and HIST_PREC_F64ATOMIC)."""
import math

import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import assert_sums_close, check_against_oracle, edge_probe_values, gpu_fill, to_device

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


LOCATE_AXES = [
    W.fixed(100, 0.0, 1.0), W.fixed(1000, -5.0, 5.0), W.fixed(222, -1.0, 1.5),
    W.fixed(7, -0.3, 0.4), W.fixed(1, 2.0, 3.0), W.fixed(100000, 0.0, 300.0),
    W.fixed(64, -1e-300, 1e-300), W.fixed(50, 1e15, 1e15 + 1.0), W.fixed(3, -1e300, 1e300),
    W.variable(W.log_edges(500, 0.0, 3.0)), W.variable([-3.0, -1.0, -0.0, 0.5, 10.0]),
    W.variable(np.sort(np.random.default_rng(3).normal(0, 1, 20001))),
]


@pytest.mark.parametrize("axis", LOCATE_AXES, ids=lambda a: f"{a['kind']}{a.get('nbins', len(a.get('edges', [])) - 1)}")
def test_locate_edges_bit_exact(B, axis):
    """Every threshold, its neighbours, signed zeros, infinities, NaNs,
    subnormals, huge values: GPU find-bin equals the oracle's."""
    import torch
    rng = np.random.default_rng(5)
    T = B.hist_axis_thresholds(axis)
    x = edge_probe_values(axis, T, rng)
    ref = oracle.locate([axis], x.reshape(1, -1))
    h = B.Hist([axis])
    try:
        got = h.locate(to_device(x.reshape(1, -1))).cpu().numpy()
        torch.cuda.synchronize()
    finally:
        h.close()
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, f"{bad.size} mismatches, e.g. x={x[bad[:5]]!r} got {got[bad[:5]]} ref {ref[bad[:5]]}"


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("axis", LOCATE_AXES, ids=lambda a: f"{a['kind']}{a.get('nbins', len(a.get('edges', [])) - 1)}")
def test_fill_edges_bit_exact(B, axis, weighted):
    """The same probes through hist_fill_bulk: the fill kernels carry their
    own locate (compiled per locate mode, the FP32 estimate gated on the
    double-word range, the specialised bucket kernel for weighted fills), so
    every threshold, its neighbouring keys and the special values go through
    it too, in shuffled order; counts bit-exact against the oracle, and the
    unit-weight bins equal to the counts."""
    rng = np.random.default_rng(6)
    T = B.hist_axis_thresholds(axis)
    x = edge_probe_values(axis, T, rng)
    x = x[rng.permutation(x.size)]
    w = rng.uniform(0.5, 1.5, x.size) if weighted else None
    ref = oracle.fill([axis], x.reshape(1, -1), w)
    bins, stats, counts = gpu_fill([axis], x, w, flags=B.HIST_TRACK_COUNTS)
    bad = np.flatnonzero(counts != ref.counts)
    assert bad.size == 0, f"{bad.size} bins with other counts, e.g. {bad[:5]}: {counts[bad[:5]]} vs {ref.counts[bad[:5]]}"
    if not weighted:
        assert np.array_equal(bins, ref.counts.astype(np.float64))
    assert stats[0] == x.size


def test_locate_nd_bit_exact(B):
    rng = np.random.default_rng(8)
    axes = [W.fixed(30, -2.0, 2.0), W.variable(np.sort(rng.uniform(-3, 3, 41))), W.fixed(5, 0.0, 1.0)]
    n = 100_003
    v = np.empty((3, n))
    v[0] = rng.normal(0, 1.3, n)
    v[1] = rng.normal(0, 2, n)
    v[2] = rng.uniform(-0.2, 1.2, n)
    v[:, :7] = [[math.nan, -0.0, math.inf, -2.0, 2.0, 1.9999999999999998, -math.inf]] * 3
    ref = oracle.locate(axes, v)
    h = B.Hist(axes)
    try:
        got = h.locate(to_device(v)).cpu().numpy()
    finally:
        h.close()
    assert np.array_equal(got, ref)


def test_cfg1_unit_weights_full_size(B):
    """1D, 100 fixed bins on [0,1), 2^20 values on [-0.1, 1.1): counts and
    unit-weight bins bit-exact, statistics within tolerance."""
    wl = W.cfg1()
    ref = oracle.fill(wl.axes, wl.values)
    bins, stats, counts = gpu_fill(wl.axes, wl.values)
    check_against_oracle(wl.axes, wl.values, None, bins, stats, counts, ref, what="cfg1")
    assert counts.sum() == wl.n and counts[0] > 0 and counts[-1] > 0


SMALL = [("2a", 1_000_003), ("2b", 1_000_003), ("3a", 300_001), ("3b", 300_001)]


@pytest.mark.parametrize("name,n", SMALL)
@pytest.mark.parametrize("prec", ["fp64", "f64atomic"])
def test_weighted_configs_small(B, name, n, prec):
    wl = W.CONFIGS[name](n=n)
    flags = B.HIST_TRACK_COUNTS | (B.HIST_PREC_F64ATOMIC if prec == "f64atomic" else B.HIST_PREC_FP64)
    ref = oracle.fill(wl.axes, wl.values, wl.weights, threads=4)
    bins, stats, counts = gpu_fill(wl.axes, wl.values, wl.weights, flags=flags)
    check_against_oracle(wl.axes, wl.values, wl.weights, bins, stats, counts, ref, RTOL, RTOL,
                         what=f"cfg{name} {prec}")


@pytest.mark.parametrize("name", ["1", "2a", "2b", "3b"])
def test_fills_accumulate(B, name):
    """Several fills of slices equal one fill of the whole (Sec. 3.3: running
    sums combine with the previous bulk); the fixed-point bins are exact
    integers, so they are bit-identical however the events are split."""
    wl = W.CONFIGS[name](n=200_001)
    flags = B.HIST_TRACK_COUNTS
    one = gpu_fill(wl.axes, wl.values, wl.weights, flags=flags, chunks=1)
    many = gpu_fill(wl.axes, wl.values, wl.weights, flags=flags, chunks=7)
    assert np.array_equal(one[0], many[0])
    assert np.array_equal(one[2], many[2])
    ref = oracle.fill(wl.axes, wl.values, wl.weights)
    check_against_oracle(wl.axes, wl.values, wl.weights, *many, ref, RTOL, RTOL, what=f"cfg{name} chunks")


@pytest.mark.parametrize("n", [0, 1, 2, 3, 33, 1025, 4099])
def test_ragged_sizes(B, n):
    rng = np.random.default_rng(n)
    axes = [W.fixed(1000, -5.0, 5.0)]
    x = rng.normal(0, 2, n).reshape(1, n)
    w = rng.uniform(0.5, 1.5, n)
    ref = oracle.fill(axes, x, w)
    bins, stats, counts = gpu_fill(axes, x, w, flags=B.HIST_TRACK_COUNTS)
    check_against_oracle(axes, x, w, bins, stats, counts, ref, RTOL, RTOL, what=f"n={n}")


def test_unaligned_columns(B):
    """Columns that are 8- but not 16-byte aligned take the scalar-load path."""
    import torch
    rng = np.random.default_rng(2)
    n = 10_001
    axes = [W.fixed(50, -3.0, 3.0), W.variable(np.linspace(-2, 2, 17))]
    v = rng.normal(0, 1.5, (2, n))
    w = rng.uniform(0.5, 1.5, n)
    buf = torch.zeros(2 * n + 1, dtype=torch.float64, device="cuda")
    buf[1:] = torch.from_numpy(v.reshape(-1)).cuda()
    wbuf = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    wbuf[1:] = torch.from_numpy(w).cuda()
    h = B.Hist(axes, B.HIST_TRACK_COUNTS)
    try:
        B.hist_fill_bulk(h.h, buf.data_ptr() + 8, wbuf.data_ptr() + 8, n)
        bins, stats = h.result()
        counts = h.counts()
    finally:
        h.close()
    ref = oracle.fill(axes, v, w)
    check_against_oracle(axes, v, w, bins, stats, counts, ref, RTOL, RTOL, what="unaligned")


def test_misaligned_pointer_rejected(B):
    import torch
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    h = B.Hist([W.fixed(10, 0.0, 1.0)])
    try:
        with pytest.raises(B.HistError) as e:
            B.hist_fill_bulk(h.h, buf.data_ptr() + 4, None, 8)
        assert e.value.code == B.HIST_ERR_ALIGN
        with pytest.raises(B.HistError) as e:
            B.hist_fill_bulk(h.h, 0, None, 8)
        assert e.value.code == B.HIST_ERR_ARG
        with pytest.raises(B.HistError) as e:
            B.hist_fill_bulk(h.h, buf.data_ptr(), None, -1)
        assert e.value.code == B.HIST_ERR_ARG
    finally:
        h.close()


def test_specials_and_stat_overflows(B):
    """NaN / inf coordinates, NaN / inf / zero / out-of-window weights, with
    and without HIST_STAT_OVERFLOWS."""
    rng = np.random.default_rng(4)
    n = 5000
    x = rng.normal(0, 2, n)
    w = rng.uniform(0.5, 1.5, n)
    x[:12] = [math.nan, -math.nan, math.inf, -math.inf, 0.0, -0.0, 5e-324, 1e300, -1e300, 4.999999999999999, -5.0, 5.0]
    w[20:30] = [0.0, -0.0, 1e-30, 1e30, 300.0, -7.5, 2.0 ** -9, 2.0 ** 8, 2.0 ** -8, -(2.0 ** 8) + 1]
    axes = [W.fixed(100, -5.0, 5.0)]
    for so in (False, True):
        flags = B.HIST_TRACK_COUNTS | (B.HIST_STAT_OVERFLOWS if so else 0)
        ref = oracle.fill(axes, x.reshape(1, -1), w, stat_overflows=so)
        bins, stats, counts = gpu_fill(axes, x, w, flags=flags)
        if not so:
            check_against_oracle(axes, x, w, bins, stats, counts, ref, RTOL, RTOL, what="specials")
        else:
            # the NaN / inf coordinates make the statistics non-finite
            assert np.array_equal(counts, ref.counts)
            assert np.isnan(stats[3]) and np.isnan(ref.stats_acc[3])
    # NaN weight poisons its bin only
    w2 = w.copy()
    w2[100] = math.nan
    ref = oracle.fill(axes, x.reshape(1, -1), w2)
    bins, stats, counts = gpu_fill(axes, x, w2, flags=B.HIST_TRACK_COUNTS)
    g = ref.counts.nonzero()[0]
    assert np.isnan(bins[oracle.locate(axes, x[100:101].reshape(1, 1))[0]])
    assert np.array_equal(np.isnan(bins), np.isnan(ref.bins_acc))


@pytest.mark.parametrize("p_neg,wmax", [(0.5, 1.5), (0.9, 1.5), (0.5, 255.0)])
def test_signed_weights_few_bins(B, p_neg, wmax):
    """Weights of both signs (mostly negative ones in one case) piled into
    three shared bins: the carry and borrow chains of the fixed-point words
    run thousands of times per block, totals go negative, and the bins are
    identical whether the events come in one fill or in seven (every weight
    lies in the fixed-point window, so the sums are exact)."""
    rng = np.random.default_rng(12)
    n = 2_000_003
    x = rng.uniform(-0.5, 3.5, n)  # the flows too
    mag = rng.uniform(2.0 ** -8, wmax, n)
    w = np.where(rng.random(n) < p_neg, -mag, mag)
    axes = [W.fixed(3, 0.0, 3.0)]
    ref = oracle.fill(axes, x.reshape(1, -1), w, threads=4)
    one = gpu_fill(axes, x, w, flags=B.HIST_TRACK_COUNTS)
    many = gpu_fill(axes, x, w, flags=B.HIST_TRACK_COUNTS, chunks=7)
    check_against_oracle(axes, x, w, *one, ref, RTOL, RTOL, what="signed weights")
    assert np.array_equal(one[0], many[0])
    assert np.array_equal(one[2], many[2])


def test_unit_and_weighted_fills_mix(B):
    """A unit-weight fill followed by a weighted fill of the same histogram."""
    import torch
    rng = np.random.default_rng(9)
    axes = [W.fixed(40, -2.0, 2.0)]
    x1 = rng.normal(0, 1, 3001).reshape(1, -1)
    x2 = rng.normal(0, 1, 2001).reshape(1, -1)
    w2 = rng.uniform(0.5, 1.5, 2001)
    acc = oracle.Accumulator(axes)
    acc.fill(x1)
    acc.fill(x2, w2)
    ref = acc.result()
    h = B.Hist(axes, B.HIST_TRACK_COUNTS)
    try:
        h.fill(to_device(x1))
        h.fill(to_device(x2), to_device(w2))
        bins, stats = h.result()
        counts = h.counts()
    finally:
        h.close()
    assert np.array_equal(counts, ref.counts)
    check_against_oracle(axes, None, w2, bins, stats, counts, ref, RTOL, RTOL, what="mixed")


def test_result_idempotent_and_reset(B):
    wl = W.cfg2a(n=50_000)
    h = B.Hist(wl.axes, B.HIST_TRACK_COUNTS)
    try:
        h.fill(to_device(wl.values), to_device(wl.weights))
        a = h.result()
        b = h.result()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        h.reset()
        z = h.result()
        assert not z[0].any() and not z[1].any()
        assert not h.counts().any()
    finally:
        h.close()


@pytest.mark.parametrize("name", ["2a", "2b", "3a", "3b"])
def test_weighted_configs_full_size(B, name):
    """The full 1e8-event configurations in the default launch configuration,
    against the chunk-parallel oracle on all host cores."""
    import os
    wl = W.CONFIGS[name]()
    ref = oracle.fill(wl.axes, wl.values, wl.weights, threads=os.cpu_count() or 4)
    bins, stats, counts = gpu_fill(wl.axes, wl.values, wl.weights, flags=B.HIST_TRACK_COUNTS)
    check_against_oracle(wl.axes, wl.values, wl.weights, bins, stats, counts, ref, RTOL, RTOL,
                         what=f"cfg{name} full")


@pytest.mark.parametrize("weighted", [False, True])
def test_zero_and_tiny_coordinates(B, weighted):
    """In-range coordinates outside the double-word range (exact zeros,
    subnormals, tiny values) take the binary64 statistics path; with unit
    weights sum w^2 must still equal the in-range entry count."""
    rng = np.random.default_rng(12)
    n = 20_001
    x = rng.normal(0, 0.5, n)
    x[::3] = 0.0
    x[1::7] = -0.0
    x[2::11] = 1e-300
    x[3::13] = -5e-324
    x[4::17] = 3e-13
    axes = [W.fixed(10, -1.0, 1.0)]
    w = rng.uniform(0.5, 1.5, n) if weighted else None
    ref = oracle.fill(axes, x.reshape(1, -1), w)
    bins, stats, counts = gpu_fill(axes, x, w, flags=B.HIST_TRACK_COUNTS)
    check_against_oracle(axes, x, w, bins, stats, counts, ref, RTOL, RTOL, what=f"zeros weighted={weighted}")


@pytest.mark.parametrize("name,n", [("2a", 2_000_003), ("2b", 2_000_003), ("3b", 1_000_001), ("1", 1 << 20)])
def test_fp32c_within_tolerance(B, name, n):
    """HIST_PREC_FP32C (FP32 compensated shared-memory partials): counts
    exact; every bin within 1e-12 of its sum |w| -- the tolerance of the
    binary64 paths.  The stated bound per bin,
        |err| <= 2^-48 ((m + 1)^2 + 1) A + B 2^-53 A
    (m = the bin's entries in one block, A = sum |w| of the bin, B blocks),
    is a worst case that reaches 1e-12 A near 14 entries per bin and block;
    the errors measured are near 1e-15 A.  A compensation that lost the
    TwoSum error term would be off by about 2^-24 of a block's partial per
    entry, orders of magnitude above the tolerance
    (tests/test_precision_model.py shows both on a CPU model of the same
    arithmetic).  Statistics (double-word path) within 1e-12 of sum
    |term|."""
    wl = W.CONFIGS[name](n=n)
    w = wl.weights if wl.weights is not None else np.random.default_rng(3).uniform(0.5, 1.5, n)
    flags = B.HIST_TRACK_COUNTS | B.HIST_PREC_FP32C
    ref = oracle.fill(wl.axes, wl.values, w, threads=4)
    bins, stats, counts = gpu_fill(wl.axes, wl.values, w, flags=flags)
    assert np.array_equal(counts, ref.counts)
    rel = assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, f"cfg{name} FP32C bins")
    print(f"cfg{name} FP32C: max |err| / sum|w| per bin = {rel:.3g}")
    assert stats[0] == ref.stats_acc[0]
    assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"cfg{name} FP32C stats")


@pytest.mark.parametrize("name", ["1", "2a", "2b"])
@pytest.mark.parametrize("specials", [False, True])
def test_count_and_plain_kernel_variants_agree(B, name, specials):
    """1D fills with and without per-bin counts run different compiled
    kernel variants (affine, bucket-map and specialised bucket locates):
    the exact bins are bit-identical and both match the oracle.  With
    specials, a sprinkling of events takes the rare per-event paths (NaN,
    infinities, zeros, negative and tiny coordinates; zero and negative
    weights, weights at the ends of the fixed-point window); n is odd (the
    last event too).  (Weights outside the window take binary64 atomics,
    whose sums depend on their order: other tests hold those to the
    oracle's tolerance.)"""
    wl = W.CONFIGS[name](n=1_000_001)
    x = np.array(wl.values, copy=True)
    w = None if wl.weights is None else np.array(wl.weights, copy=True)
    if specials:
        rng = np.random.default_rng(17)
        idx = rng.choice(x.shape[1], 3000, replace=False)
        x[0, idx[:1500]] = rng.choice([math.nan, math.inf, -math.inf, 0.0, -0.0, -3.0, 1e-300, 5e-324, 2e12, -0.5],
                                      1500)
        x[0, -1] = math.nan
        if w is not None:
            w[idx[1000:]] = rng.choice([0.0, -0.75, -2.0, 2.0 ** -8, 255.0, -(2.0 ** -8)], 2000)
    plain = gpu_fill(wl.axes, x, w)
    counted = gpu_fill(wl.axes, x, w, flags=B.HIST_TRACK_COUNTS)
    assert np.array_equal(plain[0], counted[0]), "bins differ between the kernel variants"
    assert plain[1][0] == counted[1][0] == x.shape[1]
    ref = oracle.fill(wl.axes, x, w, threads=4)
    check_against_oracle(wl.axes, x, w, *plain, ref, RTOL, RTOL, what=f"no counts cfg{name}")
    check_against_oracle(wl.axes, x, w, *counted, ref, RTOL, RTOL, what=f"counts cfg{name}")


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("axis", [W.fixed(1000, -5.0, 5.0), W.variable(W.log_edges(500, 0.0, 3.0))],
                         ids=["fixed1000", "log500"])
def test_empty_and_tiny_fills(B, axis, weighted):
    """Fills of 0 events change nothing, through every fill entry point
    (device bulk, host pipeline, Filter/Define, batch); fills of 1, 2, 3
    and 5 events (fewer than one thread's pair, an odd last event, flows
    and NaN among them) then accumulate exactly as the oracle's fill of
    the same events in the same order."""
    import torch
    rng = np.random.default_rng(31)
    xs = np.array([-7.0, 0.5, 3.0, math.nan, 1200.0, 0.999, 25.0, -0.0, 1.0, 999.9, 12.5])
    ws = rng.uniform(0.5, 1.5, xs.size) if weighted else None
    h = B.Hist([axis])
    hb = B.Hist([axis])
    batch = None
    try:
        empty = torch.empty(0, dtype=torch.float64, device="cuda")
        h.fill(empty, empty if weighted else None)
        h.fill_host(torch.empty(0, dtype=torch.float64), torch.empty(0, dtype=torch.float64) if weighted else None)
        h.fill_columns([empty], [(B.HIST_DEF_COL, 0, 0)], [], empty if weighted else None)
        batch = B.Batch([hb], [0])
        batch.fill([empty], empty if weighted else None)
        torch.cuda.synchronize()
        for hh in (h, hb):
            bins, stats = hh.result()
            assert not np.any(bins) and not np.any(stats), "an empty fill changed the histogram"
        done = 0
        for m in (1, 2, 3, 5):
            xd = to_device(xs[done:done + m].copy())
            wd = None if ws is None else to_device(ws[done:done + m].copy())
            h.fill(xd, wd)
            batch.fill([xd], wd)
            done += m
        torch.cuda.synchronize()
        ref = oracle.fill([axis], xs[:done].reshape(1, -1), None if ws is None else ws[:done])
        for what, hh in (("bulk", h), ("batch", hb)):
            bins, stats = hh.result()
            check_against_oracle([axis], xs[:done], None if ws is None else ws[:done], bins, stats, None, ref,
                                 what=f"tiny fills ({what})")
    finally:
        if batch is not None:
            batch.close()
        h.close()
        hb.close()


@pytest.mark.parametrize("n", [300_007, 6_000_001], ids=["flush_in_fill", "reduce_kernel"])
def test_statistics_bit_reproducible(B, n):
    """The plain fill's statistics do not depend on the run: each thread
    adds its events in a fixed order, blocks combine their threads with a
    fixed tree, and the block partials are added in block order -- by the
    fill's last block for small fills, by the reduce kernel for large ones.
    Two fills of the same events into fresh histograms give the same
    statistics bit for bit (and the same bins)."""
    import torch
    wl = W.cfg2a(n=n)
    x = to_device(wl.values[0])
    w = to_device(wl.weights)
    got = []
    for _ in range(2):
        h = B.Hist(wl.axes)
        try:
            h.fill(x, w)
            torch.cuda.synchronize()
            got.append(h.result())
        finally:
            h.close()
    (b0, s0), (b1, s1) = got
    assert np.array_equal(b0, b1)
    assert np.array_equal(s0.view(np.uint64), s1.view(np.uint64)), f"statistics differ: {s0} {s1}"
    ref = oracle.fill(wl.axes, wl.values, wl.weights)
    check_against_oracle(wl.axes, wl.values, wl.weights, b0, s0, None, ref, what="reproducible fill")
