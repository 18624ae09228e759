"""The batched fill: every histogram of a batch filled from one event stream
in one launch must match the CPU oracle filled one histogram at a time
(counts exact, sums within 1e-12 of sum |term|)."""
import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import assert_sums_close, to_device

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


@pytest.mark.parametrize("weighted", [True, False])
@pytest.mark.parametrize("learned", [False, True])
def test_batch_matches_oracle(B, weighted, learned):
    bw = W.cfg4(n=200_003)
    hists = [B.Hist([ax]) for ax in bw.axes]
    batch = None
    try:
        if learned:
            for h, ax in zip(hists, bw.axes):
                if ax["kind"] == "variable":
                    h.train_locator(0)
        batch = B.Batch(hists, bw.col_of_hist)
        cols = [to_device(np.ascontiguousarray(bw.columns[c])) for c in range(3)]
        w = to_device(bw.weights) if weighted else None
        batch.fill(cols, w)
        _check(bw, hists, bw.weights if weighted else None, f"w={weighted} learned={learned}")
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
