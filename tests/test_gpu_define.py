"""Fused Filter/Define fill (hist_fill_columns) against the oracle: the
paper's RDataFrame example (rows with x nonzero kept, r2 = x^2 + y^2 defined
per row, r2 histogrammed) and 2D and weighted variants, with zeros, signed zeros,
NaN and infinities in the source columns.  Counts exact; weighted sums and
statistics within 1e-12 of sum |term|; the entry count is the number of
rows that pass the filters."""
import math

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


def _columns(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1.5, n)
    y = rng.normal(0, 1.5, n)
    z = rng.uniform(-1, 1, n)
    x[::10] = 0.0
    x[5::97] = -0.0
    y[3::101] = math.nan
    z[7::103] = math.inf
    return [x, y, z], rng.uniform(0.5, 1.5, n)


CASES = [
    ("paper_r2_fixed", [W.fixed(200, 0.0, 20.0)], [(0, 1, 1)], [(0, 0, 0.0)], False),
    ("r2_log_weighted", [W.variable(W.log_edges(300, -2.0, 2.0))], [(1, 0, 1)], [(0, 0, 0.0)], True),
    ("hypot_2d_weighted", [W.fixed(100, 0.0, 5.0), W.fixed(50, -3.0, 3.0)], [(2, 0, 1), (5, 0, 1)],
     [(0, 0, 0.0), (2, 2, 0.5)], True),
    ("mul_add_no_filter", [W.fixed(64, -4.0, 4.0), W.fixed(64, -4.0, 4.0)], [(3, 0, 2), (4, 1, 2)], [], False),
]


@pytest.mark.parametrize("name,axes,defines,filters,weighted", CASES, ids=[c[0] for c in CASES])
def test_fill_columns_matches_oracle(B, name, axes, defines, filters, weighted):
    import torch
    n = 500_003
    cols, w = _columns(n, 17)
    if not weighted:
        w = None
    h = B.Hist(axes, B.HIST_TRACK_COUNTS)
    try:
        h.fill_columns([to_device(c) for c in cols], defines, filters, to_device(w))
        torch.cuda.synchronize()
        bins, stats = h.result()
        counts = h.counts()
    finally:
        h.close()
    mask, vals = oracle.define_filter(cols, defines, filters)
    v = np.ascontiguousarray(vals[:, mask])
    ww = None if w is None else np.ascontiguousarray(w[mask])
    ref = oracle.fill(axes, v, ww)
    assert np.array_equal(counts, ref.counts)
    assert stats[0] == float(mask.sum())
    if w is None:
        assert np.array_equal(bins, ref.counts.astype(np.float64))
    else:
        assert_sums_close(bins, ref.bins_acc, ref.bins_abs, RTOL, f"{name} bins")
    assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], RTOL, f"{name} stats")


def test_fill_columns_rejects_bad_arguments(B):
    x = to_device(np.zeros(8))
    h = B.Hist([W.fixed(4, 0.0, 1.0)])
    h3 = B.Hist([W.fixed(4, 0.0, 1.0)] * 3)
    try:
        with pytest.raises(B.HistError) as e:
            h.fill_columns([x], [(1, 0, 3)])  # column 3 of 1
        assert e.value.code == B.HIST_ERR_ARG
        with pytest.raises(B.HistError) as e:
            h.fill_columns([x], [(9, 0, 0)])  # unknown define
        assert e.value.code == B.HIST_ERR_ARG
        with pytest.raises(B.HistError) as e:
            h3.fill_columns([x], [(0, 0, 0)] * 3)
        assert e.value.code == B.HIST_ERR_UNSUPPORTED
    finally:
        h.close()
        h3.close()
