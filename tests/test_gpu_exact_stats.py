"""HIST_STATS_EXACT: the 1D statistics equal the correctly rounded exact sums
of their rounded terms (the oracle's exact_stats), bit for bit, and are the
same bits however the events are split into fills or ordered -- with tiny
and huge coordinates and weights (the escape path), negative weights, and
NaN and infinite weights."""
import math

import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import gpu_fill

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


def _same(a, b):
    return (math.isnan(a) and math.isnan(b)) or a == b


@pytest.mark.parametrize("name,n", [("2a", 1_000_003), ("2b", 1_000_003), ("1", 1 << 20)])
def test_exact_stats_bit_exact(B, name, n):
    wl = W.CONFIGS[name](n=n)
    flags = B.HIST_STATS_EXACT
    want = oracle.exact_stats(wl.axes, wl.values, wl.weights)
    one = gpu_fill(wl.axes, wl.values, wl.weights, flags=flags)
    many = gpu_fill(wl.axes, wl.values, wl.weights, flags=flags, chunks=13)
    perm = np.random.default_rng(1).permutation(n)
    v = np.ascontiguousarray(wl.values[:, perm])
    w = None if wl.weights is None else np.ascontiguousarray(wl.weights[perm])
    shuffled = gpu_fill(wl.axes, v, w, flags=flags)
    for k in range(4):
        assert one[1][1 + k] == want[k], f"cfg{name} stat {1 + k}: {one[1][1 + k]!r} vs exact {want[k]!r}"
        assert many[1][1 + k] == one[1][1 + k]
        assert shuffled[1][1 + k] == one[1][1 + k]


def test_exact_stats_escape_and_specials(B):
    rng = np.random.default_rng(4)
    n = 300_001
    axes = [W.fixed(50, -1e6, 1e6)]
    x = rng.normal(0, 1e5, n)
    x[::17] = rng.normal(0, 1e-250, x[::17].shape[0])  # terms far below the fast window
    w = rng.uniform(-2, 2, n) * 10.0 ** rng.integers(-30, 30, n)  # wide weights: some escape upwards
    want = oracle.exact_stats(axes, x, w)
    got = gpu_fill(axes, x.reshape(1, -1), w, flags=B.HIST_STATS_EXACT)[1]
    for k in range(4):
        assert got[1 + k] == want[k], f"stat {1 + k}: {got[1 + k]!r} vs exact {want[k]!r}"
    w2 = w.copy()
    w2[5] = math.nan
    w2[7] = math.inf
    want2 = oracle.exact_stats(axes, x, w2)
    got2 = gpu_fill(axes, x.reshape(1, -1), w2, flags=B.HIST_STATS_EXACT)[1]
    assert all(_same(got2[1 + k], want2[k]) for k in range(4)), (got2, want2)


@pytest.mark.parametrize("name,n", [("3a", 1_000_003), ("3b", 700_001)])
def test_exact_stats_nd_bit_exact(B, name, n):
    """2D and 3D: all 7 / 11 statistics (ROOT's TH2/TH3 term sets) bit for
    bit equal to the oracle's correctly rounded exact sums, and the same
    bits for fills split in 7 and for shuffled events."""
    wl = W.CONFIGS[name](n=n)
    want = oracle.exact_stats(wl.axes, wl.values, wl.weights)
    flags = B.HIST_STATS_EXACT
    one = gpu_fill(wl.axes, wl.values, wl.weights, flags=flags)
    many = gpu_fill(wl.axes, wl.values, wl.weights, flags=flags, chunks=7)
    perm = np.random.default_rng(2).permutation(n)
    shuffled = gpu_fill(wl.axes, np.ascontiguousarray(wl.values[:, perm]), np.ascontiguousarray(wl.weights[perm]),
                        flags=flags)
    assert len(want) == len(one[1]) - 1
    for k in range(len(want)):
        assert one[1][1 + k] == want[k], f"cfg{name} stat {1 + k}: {one[1][1 + k]!r} vs exact {want[k]!r}"
        assert many[1][1 + k] == one[1][1 + k]
        assert shuffled[1][1 + k] == one[1][1 + k]


def test_exact_stats_nd_escape_unit_and_flows(B):
    """3D with unit weights, coordinates far outside the fast window (the
    escape limbs), and HIST_STAT_OVERFLOWS (flow entries in the sums)."""
    rng = np.random.default_rng(5)
    n = 200_001
    axes = [W.fixed(20, -1e4, 1e4), W.variable(np.sort(rng.uniform(-3, 3, 30))), W.fixed(8, 0.0, 1.0)]
    v = np.stack([rng.normal(0, 3e3, n), rng.normal(0, 2, n), rng.uniform(-0.2, 1.2, n)])
    v[0, ::13] = rng.normal(0, 1e-200, v[0, ::13].shape[0])
    for so in (False, True):
        flags = B.HIST_STATS_EXACT | (B.HIST_STAT_OVERFLOWS if so else 0)
        want = oracle.exact_stats(axes, v, None, stat_overflows=so)
        got = gpu_fill(axes, v, None, flags=flags)[1]
        for k in range(len(want)):
            assert got[1 + k] == want[k], f"overflows={so} stat {1 + k}: {got[1 + k]!r} vs exact {want[k]!r}"


def test_exact_stats_rejected_where_unsupported(B):
    import torch
    h = B.Hist([W.fixed(4, 0.0, 1.0)], B.HIST_STATS_EXACT)
    try:
        x = torch.zeros(16, dtype=torch.float64, device="cuda")
        with pytest.raises(B.HistError) as e:
            h.fill_columns([x], [(B.HIST_DEF_COL, 0, 0)])
        assert e.value.code == B.HIST_ERR_UNSUPPORTED
        with pytest.raises(B.HistError) as e:
            B.Batch([h], [0])
        assert e.value.code == B.HIST_ERR_UNSUPPORTED
    finally:
        h.close()
