"""The batched fill: every histogram of a batch filled from one event stream
in one launch must match the CPU oracle filled one histogram at a time
(counts exact, sums within 1e-12 of sum |term|), under each privatisation
strategy (wide: per-block shared bins for the small histograms, global
atomics for the rest; sliced: every bin in shared memory, large histograms
cut into fragments across blocks; partitioned: each column's events
partitioned by coordinate range, every member's bins of a range in one
block's shared memory)."""
import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import assert_sums_close, edge_probe_values, to_device

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


def _check(bw, hists, weights, what):
    cols = bw.columns
    for i, (h, ax, c) in enumerate(zip(hists, bw.axes, bw.col_of_hist)):
        bins, stats = h.result()
        ref = oracle.fill([ax], cols[c].reshape(1, -1), weights)
        if weights is None:
            assert np.array_equal(bins, ref.counts.astype(np.float64)), f"{what} hist {i}"
        else:
            assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, f"{what} hist {i} bins")
        assert stats[0] == ref.stats_acc[0]
        assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"{what} hist {i} stats")


STRATEGIES = {"wide": 1 << 1, "sliced": 1 << 2}


@pytest.mark.parametrize("strategy", ["wide", "sliced"])
@pytest.mark.parametrize("weighted", [True, False])
@pytest.mark.parametrize("learned", [False, True])
def test_batch_matches_oracle(B, strategy, weighted, learned):
    bw = W.cfg4(n=200_003)
    hists = [B.Hist([ax]) for ax in bw.axes]
    batch = None
    try:
        if learned:
            for h, ax in zip(hists, bw.axes):
                if ax["kind"] == "variable":
                    h.train_locator(0)
        batch = B.Batch(hists, bw.col_of_hist, STRATEGIES[strategy])
        cols = [to_device(np.ascontiguousarray(bw.columns[c])) for c in range(3)]
        w = to_device(bw.weights) if weighted else None
        batch.fill(cols, w)
        _check(bw, hists, bw.weights if weighted else None, f"{strategy} w={weighted} learned={learned}")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


def test_batch_graph_tune_and_accumulate(B):
    """Autotuning leaves the histograms untouched; two graph-replayed fills
    accumulate like two fills."""
    bw = W.cfg4(n=100_001)
    hists = [B.Hist([ax]) for ax in bw.axes]
    batch = None
    try:
        batch = B.Batch(hists, bw.col_of_hist, B.HIST_BATCH_GRAPH)
        cols = [to_device(np.ascontiguousarray(bw.columns[c])) for c in range(3)]
        w = to_device(bw.weights)
        rep = batch.tune(cols, w)
        assert rep["candidates"] >= 3 and rep["best_ms"] <= rep["worst_ms"]
        for h in hists:
            b0, s0 = h.result()
            assert not b0.any() and not s0.any()
        batch.fill(cols, w)
        batch.fill(cols, w)
        two_cols = np.concatenate([bw.columns, bw.columns], axis=1)
        two_w = np.concatenate([bw.weights, bw.weights])
        for i, (h, ax, c) in enumerate(zip(hists, bw.axes, bw.col_of_hist)):
            bins, stats = h.result()
            ref = oracle.fill([ax], two_cols[c].reshape(1, -1), two_w)
            assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, f"graph hist {i}")
            assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"graph stats {i}")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


def test_batch_rejects_nd_and_bad_columns(B):
    h2 = B.Hist([W.fixed(4, 0.0, 1.0), W.fixed(4, 0.0, 1.0)])
    h1 = B.Hist([W.fixed(4, 0.0, 1.0)])
    try:
        with pytest.raises(B.HistError) as e:
            B.Batch([h2], [0])
        assert e.value.code == B.HIST_ERR_UNSUPPORTED
        with pytest.raises(B.HistError) as e:
            B.Batch([h1], [7])
        assert e.value.code == B.HIST_ERR_ARG
    finally:
        h1.close()
        h2.close()


@pytest.mark.parametrize("strategy", ["wide", "sliced"])
def test_batch_edges_specials_and_odd_weights(B, strategy):
    """Every threshold of every axis and its neighbouring doubles (so every
    fragment boundary of a cut histogram), signed zeros, infinities, NaN,
    subnormals; weights of both signs, zero, and outside the fixed-point
    window (the binary64 slow path)."""
    rng = np.random.default_rng(33)
    axes, col_of_hist = W.batch_axes(64)
    per_col = [[], [], []]
    for ax, c in zip(axes, col_of_hist):
        per_col[c].append(edge_probe_values(ax, B.hist_axis_thresholds(ax), rng, nrand=500))
    streams = [np.concatenate(v) for v in per_col]
    n = max(len(v) for v in streams)
    cols = np.empty((3, n))
    for c in range(3):
        v = np.resize(streams[c], n)
        cols[c] = v[rng.permutation(n)]
    w = rng.uniform(-2.0, 2.0, n)
    w[::97] = 0.0
    w[1::89] = 1e-5
    w[2::83] = -3e3
    bw = W.BatchWorkload("edges", axes, col_of_hist, cols, w, {})
    hists = [B.Hist([ax]) for ax in axes]
    batch = None
    try:
        batch = B.Batch(hists, col_of_hist, STRATEGIES[strategy])
        batch.fill([to_device(np.ascontiguousarray(cols[c])) for c in range(3)], to_device(w))
        _check(bw, hists, w, f"{strategy} edges")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


def test_batch_unit_weights_many_edges_tuned(B):
    """Unit weights into eight histograms of 100 .. 10^4 mixture-quantile
    edges, after tuning (whichever strategy wins): counts exact."""
    bw = W.cfg5(n=300_007, nhist=8, scale=0.01)
    hists = [B.Hist([ax]) for ax in bw.axes]
    batch = None
    try:
        batch = B.Batch(hists, bw.col_of_hist, B.HIST_BATCH_GRAPH)
        col = to_device(np.ascontiguousarray(bw.columns[0]))
        rep = batch.tune([col], None)
        assert rep["candidates"] >= 6
        batch.fill([col], None)
        _check(bw, hists, None, f"tuned strategy {rep['strategy']}")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


def test_batch_configurations_agree_exactly(B):
    """Pinned configurations (wide at two register budgets and events per
    thread, sliced at two slice sizes, partitioned at two range sizes): the
    exact fixed-point bins are bit-identical whatever the configuration;
    statistics within tolerance."""
    bw = W.cfg4(n=150_001)
    cols = [to_device(np.ascontiguousarray(bw.columns[c])) for c in range(3)]
    w = to_device(bw.weights)
    configs = [(0, 48 << 10, 30, -1, 2, 4), (0, 96 << 10, 30, -1, 4, 2), (1, 96 << 10, 30, -1, 2, 4),
               (1, 200 << 10, 120, 0, 2, 4), (2, 24 << 10, 30, -1, 2, 4), (2, 100 << 10, 30, -1, 2, 4)]
    results = []
    for cfg in configs:
        hists = [B.Hist([ax]) for ax in bw.axes]
        batch = None
        try:
            batch = B.Batch(hists, bw.col_of_hist)
            info = batch.configure(*cfg)
            assert info["strategy"] == cfg[0]
            batch.fill(cols, w)
            results.append([h.result() for h in hists])
        finally:
            if batch is not None:
                batch.close()
            for h in hists:
                h.close()
    for r in results[1:]:
        for i, ((b0, s0), (b1, s1)) in enumerate(zip(results[0], r)):
            assert np.array_equal(b0, b1), f"hist {i} bins differ between configurations"
            ref = oracle.fill([bw.axes[i]], bw.columns[bw.col_of_hist[i]].reshape(1, -1), bw.weights)
            assert_sums_close(s1[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"hist {i} stats")


def test_batch_sliced_pacing_window_does_not_change_bins(B):
    """The sliced strategy's blocks pace themselves (a bounded wait every 16
    tiles until every slice has passed the tile a window back; the waits of
    one block in one launch are capped in total).  The tightest window the
    configuration allows, on a fill long enough (8e6 events, ~3900 tiles)
    for the cap to be spent, the default window and no pacing at all give
    bit-identical exact bins, equal to the oracle's for unit weights: the
    pacing only orders work for L2 locality."""
    import torch
    rng = np.random.default_rng(81)
    bw = W.cfg4(n=10)
    n = 8_000_000
    cols_h = [rng.exponential(30.0, n), rng.uniform(-np.pi, np.pi, n), rng.normal(0.0, 2.5, n)]
    cols = [to_device(c) for c in cols_h]
    w = rng.uniform(0.5, 1.5, n)
    wd = to_device(w)
    results = {}
    for pace in (1, -1, 0):
        for weighted in (False, True):
            hists = [B.Hist([ax]) for ax in bw.axes]
            batch = None
            try:
                batch = B.Batch(hists, bw.col_of_hist)
                assert batch.configure(1, 96 << 10, 30, pace, 2, 4)["strategy"] == 1
                batch.fill(cols, wd if weighted else None)
                torch.cuda.synchronize()
                results[(pace, weighted)] = [h.result()[0] for h in hists]
            finally:
                if batch is not None:
                    batch.close()
                for h in hists:
                    h.close()
    for weighted in (False, True):
        base = results[(0, weighted)]
        for pace in (1, -1):
            for i, (a, b) in enumerate(zip(base, results[(pace, weighted)])):
                assert np.array_equal(a, b), f"hist {i}: pace {pace} changed the bins (weighted={weighted})"
    for i in (0, 21, 42, 63):  # unit-weight bins against the oracle
        ref = oracle.fill([bw.axes[i]], cols_h[bw.col_of_hist[i]].reshape(1, -1), None)
        assert np.array_equal(results[(1, False)][i], ref.counts.astype(np.float64)), f"hist {i}"


def test_batch_tuned_for_unit_then_weighted_fill(B):
    """A batch tuned on a unit-weight sample keeps one word per shared bin;
    a weighted fill afterwards re-places the bins (two words) and both fills
    match the oracle."""
    bw = W.cfg4(n=120_001)
    hists = [B.Hist([ax]) for ax in bw.axes]
    batch = None
    try:
        batch = B.Batch(hists, bw.col_of_hist, B.HIST_BATCH_WIDE)
        cols = [to_device(np.ascontiguousarray(bw.columns[c])) for c in range(3)]
        batch.tune(cols, None)
        batch.fill(cols, None)
        batch.fill(cols, to_device(bw.weights))
        ones = np.ones(bw.n)
        for i, (h, ax, c) in enumerate(zip(hists, bw.axes, bw.col_of_hist)):
            bins, stats = h.result()
            x2 = np.concatenate([bw.columns[c], bw.columns[c]]).reshape(1, -1)
            w2 = np.concatenate([ones, bw.weights])
            ref = oracle.fill([ax], x2, w2)
            assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, f"hist {i} bins")
            assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"hist {i} stats")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


@pytest.mark.parametrize("plan", ["tuned", "wide", "partitioned"])
@pytest.mark.parametrize("odd", [False, True])
def test_batch_fp32c_matches_oracle(B, odd, plan):
    """A batch whose members are all booked HIST_PREC_FP32C runs the FP32
    compensated form (shared FP32 hi/lo bins with TwoSum on the atomic's old
    value; in the wide strategy binary64 atomics for the large members):
    bins and statistics within 1e-12 of the oracle's sum of |terms|, after
    tuning and with the wide and partitioned strategies pinned.  With odd
    weights (zero, negative, tiny, huge) the events outside the double-word
    range take the binary64 path."""
    bw = W.cfg4(n=200_003)
    w = np.array(bw.weights, copy=True)
    if odd:
        rng = np.random.default_rng(44)
        w[::53] = 0.0
        w[1::47] = -rng.uniform(0.5, 1.5, w[1::47].shape[0])
        w[2::61] = 1e-13
        w[3::67] = 3e14
    hists = [B.Hist([ax], B.HIST_PREC_FP32C) for ax in bw.axes]
    batch = None
    try:
        with pytest.raises(B.HistError) as e:
            B.Batch(hists, bw.col_of_hist, STRATEGIES["sliced"])
        assert e.value.code == B.HIST_ERR_UNSUPPORTED
        batch = B.Batch(hists, bw.col_of_hist, B.HIST_BATCH_GRAPH)
        cols = [to_device(np.ascontiguousarray(bw.columns[c])) for c in range(3)]
        if plan == "tuned":
            assert batch.tune(cols, to_device(w))["strategy"] in (0, 2)
        elif plan == "wide":
            assert batch.configure(0, 48 << 10, 30, -1, 2, 4)["strategy"] == 0
        else:
            assert batch.configure(2, 48 << 10, 30, -1, 2, 4)["strategy"] == 2
        batch.fill(cols, to_device(w))
        worst = 0.0
        for i, (h, ax, c) in enumerate(zip(hists, bw.axes, bw.col_of_hist)):
            bins, stats = h.result()
            ref = oracle.fill([ax], bw.columns[c].reshape(1, -1), w)
            worst = max(worst, assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, f"fp32c hist {i} bins"))
            assert stats[0] == ref.stats_acc[0]
            assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"fp32c hist {i} stats")
        print(f"FP32C batch: max |err| / sum|w| per bin = {worst:.3g}")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


def test_batch_rejects_mixed_precision(B):
    h1 = B.Hist([W.fixed(10, 0.0, 1.0)], B.HIST_PREC_FP32C)
    h2 = B.Hist([W.fixed(10, 0.0, 1.0)])
    try:
        with pytest.raises(B.HistError) as e:
            B.Batch([h1, h2], [0, 0])
        assert e.value.code == B.HIST_ERR_UNSUPPORTED
    finally:
        h1.close()
        h2.close()


def _one_column_batch(n, seed):
    """Twelve axes of every kind (fixed, log-spaced, jittered, mixture
    quantiles; ranges inside, around and beside the data) on one column of
    values N(0.3, 3), with weights U[0.5, 1.5)."""
    rng = np.random.default_rng(seed)
    axes = []
    for i in range(12):
        kind = i % 4
        nb = int(round(10 * 10 ** (3.3 * i / 11)))
        if kind == 0:
            axes.append(W.fixed(nb, -8.0 + 0.1 * i, 9.0 - 0.2 * i))
        elif kind == 1:
            axes.append(W.variable(W.log_edges(nb, -2.0, 1.2)))
        elif kind == 2:
            axes.append(W.variable(W.jittered_edges(nb, -5.0, 5.0, rng)))
        else:
            axes.append(W.variable(W.mixture_quantile_edges(nb)))
    x = rng.normal(0.3, 3.0, n)
    w = rng.uniform(0.5, 1.5, n)
    return W.BatchWorkload("one_column", axes, [0] * len(axes), x.reshape(1, n), w, {})


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("budget", [6 << 10, 100 << 10])
def test_batch_partitioned_matches_oracle(B, weighted, budget):
    """The partitioned strategy (events partitioned by coordinate range,
    every member's bins of a range in one block's shared memory): bins and
    statistics against the oracle, with a small shared-memory budget (many
    ranges: every member cut at many range boundaries) and a large one."""
    bw = _one_column_batch(300_007, 71)
    w = bw.weights if weighted else None
    hists = [B.Hist([ax]) for ax in bw.axes]
    batch = None
    try:
        batch = B.Batch(hists, bw.col_of_hist)
        info = batch.configure(2, budget)
        assert info["strategy"] == 2 and info["slices"] >= (8 if budget < (10 << 10) else 1)
        batch.fill([to_device(np.ascontiguousarray(bw.columns[0]))], to_device(w))
        _check(bw, hists, w, f"partitioned budget={budget} w={weighted}")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


@pytest.mark.parametrize("budget", [8 << 10, 100 << 10])
@pytest.mark.parametrize("ncols", [1, 2])
@pytest.mark.parametrize("weighted", [False, True])
def test_batch_partitioned_edges_specials_and_accumulate(B, weighted, ncols, budget):
    """Every threshold of every member and its neighbouring doubles (so
    every range boundary and slice boundary), signed zeros, infinities,
    NaN, subnormals; odd weights; two fills accumulate like one of the
    concatenation (graph replay).  With two columns the members alternate
    between the probe points and the same points reversed: each column is
    partitioned and filled on its own, its statistics in its own slots.
    The small budget makes many small ranges (fills of two events per
    thread at a time); the large one ranges whose tables hold the fill to
    two blocks per SM (the kernel with four events per thread in flight)."""
    rng = np.random.default_rng(72)
    bw = _one_column_batch(10, 73)
    pts = np.concatenate([edge_probe_values(ax, B.hist_axis_thresholds(ax), rng, nrand=300) for ax in bw.axes])
    pts = pts[rng.permutation(pts.size)]
    n = pts.size
    columns = [pts, pts[::-1].copy()][:ncols]
    col_of_hist = [i % ncols for i in range(len(bw.axes))]
    w = rng.uniform(-2.0, 2.0, n) if weighted else None
    if weighted:
        w[::97] = 0.0
        w[1::89] = 1e-5
        w[2::83] = -3e3
    hists = [B.Hist([ax]) for ax in bw.axes]
    batch = None
    try:
        batch = B.Batch(hists, col_of_hist, B.HIST_BATCH_GRAPH)
        info = batch.configure(2, budget)
        assert info["strategy"] == 2
        if budget > (64 << 10):
            assert info["blocks_per_sm"] <= 2, info
        assert info["events_per_thread"] == (4 if info["blocks_per_sm"] <= 2 else 2), info
        cols = [to_device(c) for c in columns]
        wd = to_device(w)
        batch.fill(cols, wd)
        batch.fill(cols, wd)
        w2 = None if w is None else np.concatenate([w, w])
        for i, (h, ax) in enumerate(zip(hists, bw.axes)):
            bins, stats = h.result()
            c = columns[col_of_hist[i]]
            ref = oracle.fill([ax], np.concatenate([c, c]).reshape(1, -1), w2)
            if w2 is None:
                assert np.array_equal(bins, ref.counts.astype(np.float64)), f"hist {i}"
            else:
                assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, f"partitioned edges hist {i} bins")
            assert stats[0] == ref.stats_acc[0]
            assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"partitioned hist {i} stats")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


@pytest.mark.parametrize("weighted", [True, False])
@pytest.mark.parametrize("budget", [48 << 10, 100 << 10])
def test_batch_partitioned_several_columns(B, weighted, budget):
    """The 64-histogram batch (three columns of 22, 21 and 21 members, rows
    of 24 counts) with the partitioned strategy pinned: each column's
    members partitioned and filled in turn, against the oracle."""
    bw = W.cfg4(n=200_003)
    hists = [B.Hist([ax]) for ax in bw.axes]
    batch = None
    try:
        batch = B.Batch(hists, bw.col_of_hist)
        info = batch.configure(2, budget)
        assert info["strategy"] == 2 and info["slices"] >= 3
        cols = [to_device(np.ascontiguousarray(bw.columns[c])) for c in range(3)]
        w = bw.weights if weighted else None
        batch.fill(cols, to_device(w))
        _check(bw, hists, w, f"partitioned 3 columns budget={budget} w={weighted}")
    finally:
        if batch is not None:
            batch.close()
        for h in hists:
            h.close()


def test_batch_partitioned_member_limit_per_column(B):
    """At most 32 members per column: 32 on one column and 33 split over
    two columns are accepted; 33 on one column are not."""
    axes = [W.fixed(10 + i, -1.0, 1.0) for i in range(33)]  # (one range: one statistics group per column)
    hists = [B.Hist([ax]) for ax in axes]
    try:
        for members, cols, ok in ((32, [0] * 32, True), (33, [i % 2 for i in range(33)], True),
                                  (33, [0] * 33, False)):
            batch = B.Batch(hists[:members], cols)
            try:
                if ok:
                    assert batch.configure(2, 64 << 10)["strategy"] == 2
                else:
                    with pytest.raises(B.HistError) as e:
                        batch.configure(2, 64 << 10)
                    assert e.value.code == B.HIST_ERR_UNSUPPORTED
            finally:
                batch.close()
    finally:
        for h in hists:
            h.close()
