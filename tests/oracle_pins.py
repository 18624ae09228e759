"""Checks that pin the CPU oracle to facts other than its own code.

Each check raises AssertionError when the oracle disagrees with something the
paper's definitions or plain mathematics fix:

* exact rational arithmetic (``fractions.Fraction``) for the fixed-width
  formula of Sec. 3.1,
* closed forms (bin centres, dyadic axes where every binary64 step is exact),
* library routines that compute the same definition another way
  (``bisect.bisect_right`` for the binary search, ``numpy.histogram`` and
  ``numpy.bincount`` for counting and sequential summation, ``math.fsum`` for
  correctly rounded sums),
* brute force on tiny inputs (linear scans, enumerating every bin of a small
  ND histogram),
* the hand-derived cases under ``tests/golden/``.

``tests/test_oracle_pins.py`` runs them on the oracle as built, and plants
typical mistakes in a copy of the oracle's C source to show that each one is
caught by at least one check.
"""
from __future__ import annotations

import bisect
import math
import random
from fractions import Fraction

import numpy as np

import oracle
from tests import golden_io

INF = math.inf
NAN = math.nan


def exact_fixed_bin(nbins, xmin, xmax, x):
    """1 + floor(nbins (x - min) / (max - min)) in exact rational arithmetic,
    with the range tests and the x < max clamp."""
    if x < xmin:
        return 0
    if not (x < xmax):
        return nbins + 1
    q = Fraction(nbins) * (Fraction(x) - Fraction(xmin)) / (Fraction(xmax) - Fraction(xmin))
    return min(1 + math.floor(q), nbins), q


# ------------------------------------------------------------- locate ------


def check_golden_fixed():
    for nb, a, b, x, exp in golden_io.fixed_cases():
        got = oracle.find_bin_fixed(nb, a, b, x)
        assert got == exp, f"fixed golden nbins={nb} [{a},{b}) x={x!r}: {got} != {exp}"


def check_golden_variable():
    for edges, x, exp in golden_io.variable_cases():
        got = oracle.find_bin_variable(edges, x)
        assert got == exp, f"variable golden edges={edges} x={x!r}: {got} != {exp}"


def check_fixed_dyadic_exact(seed=0):
    """On [-4, 4) with 16 bins every step of the formula is exact for
    x = k * 2^-20, so the bin is exactly 1 + floor(2 (x + 4))."""
    rng = random.Random(seed)
    for _ in range(4000):
        k = rng.randint(-4 * 2 ** 20 - 100, 4 * 2 ** 20 + 100)
        x = k * 2.0 ** -20
        if x < -4:
            exp = 0
        elif x >= 4:
            exp = 17
        else:
            exp = 1 + math.floor(Fraction(2) * (Fraction(x) + 4))
        got = oracle.find_bin_fixed(16, -4.0, 4.0, x)
        assert got == exp, f"dyadic x={x!r}: {got} != {exp}"


def check_fixed_vs_rational(seed=1, ncases=3000):
    """Random axes and coordinates: the binary64 bin is within one of the
    exact rational bin, and equal to it whenever the exact quotient is not
    within 1e-9 of an integer (rounding can only matter right at an edge)."""
    rng = random.Random(seed)
    exact_hits = 0
    for _ in range(ncases):
        nb = rng.choice([1, 2, 3, 7, 10, 100, 999, 1000, 4096, 100000])
        xmin = rng.uniform(-50, 50)
        xmax = xmin + rng.choice([1e-3, 0.5, 1.0, 3.7, 10.0, 250.0])
        x = rng.uniform(xmin, xmax)
        if not (xmin <= x < xmax):
            continue
        exp, q = exact_fixed_bin(nb, xmin, xmax, x)
        got = oracle.find_bin_fixed(nb, xmin, xmax, x)
        assert abs(got - exp) <= 1, f"nb={nb} [{xmin},{xmax}) x={x!r}: {got} vs exact {exp}"
        frac = q - math.floor(q)
        if 1e-9 < frac < 1 - 1e-9:
            assert got == exp, f"nb={nb} [{xmin},{xmax}) x={x!r}: {got} vs exact {exp}"
            exact_hits += 1
    assert exact_hits > ncases // 2


def check_fixed_centres():
    """The centre of bin k lands in bin k (far from any edge)."""
    for nb, a, b in [(100, 0.0, 1.0), (1000, -5.0, 5.0), (7, 1.0, 2.0), (300, 0.0, 300.0),
                     (12345, -math.pi, math.pi), (1, -1.0, 1.0)]:
        for k in list(range(1, min(nb, 300) + 1)) + [nb]:
            c = float(Fraction(a) + (Fraction(k) - Fraction(1, 2)) * (Fraction(b) - Fraction(a)) / nb)
            got = oracle.find_bin_fixed(nb, a, b, c)
            assert got == k, f"centre of bin {k} of {nb} on [{a},{b}): got {got}"


def check_fixed_range_edges(seed=2):
    """min -> 1, below min -> 0, max -> nbins+1, the last double below max ->
    nbins (never overflow), +-inf, NaN, and -0 == +0."""
    rng = random.Random(seed)
    for _ in range(2000):
        nb = rng.randint(1, 3000)
        xmin = rng.choice([0.0, -1.0, 0.1, -5.0, 1.0, 3.0, rng.uniform(-10, 10)])
        xmax = xmin + rng.choice([1.0, 0.3, 10.0, 0.7, 2.5, 1e-3, rng.uniform(0.01, 5)])
        f = lambda x: oracle.find_bin_fixed(nb, xmin, xmax, x)  # noqa: E731
        assert f(xmin) == 1
        assert f(math.nextafter(xmin, -INF)) == 0
        assert f(xmax) == nb + 1
        assert f(math.nextafter(xmax, -INF)) == nb
        assert f(INF) == nb + 1 and f(-INF) == 0 and f(NAN) == nb + 1
    assert oracle.find_bin_fixed(10, 0.0, 1.0, -0.0) == 1
    assert oracle.find_bin_fixed(10, -1.0, 1.0, -0.0) == oracle.find_bin_fixed(10, -1.0, 1.0, 0.0) == 6


def check_fixed_monotone(seed=3):
    rng = np.random.default_rng(seed)
    for nb, a, b in [(100, 0.0, 1.0), (1000, -5.0, 5.0), (333, -0.37, 12.9)]:
        xs = np.sort(np.concatenate([rng.uniform(a - 1, b + 1, 5000),
                                     a + (b - a) * np.arange(nb + 1) / nb]))
        bins = [oracle.find_bin_fixed(nb, a, b, float(x)) for x in xs]
        assert all(u <= v for u, v in zip(bins, bins[1:])), "fixed find-bin not monotone"


def _variable_probe_points(edges, rng):
    pts = []
    for e in edges:
        pts += [e, math.nextafter(e, -INF), math.nextafter(e, INF)]
        y = e
        for _ in range(4):
            y = math.nextafter(y, -INF)
        pts.append(y)
    mids = [(u + v) / 2 for u, v in zip(edges, edges[1:])]
    pts += mids
    pts += list(rng.uniform(edges[0] - 1, edges[-1] + 1, 300))
    pts += [INF, -INF, NAN, edges[0] - 1e300 if edges[0] > -1e300 else -INF]
    return pts


def check_variable_vs_bisect_and_scan(seed=4):
    """Binary search against bisect_right (the number of edges <= x) and a
    linear scan over the bins."""
    rng = np.random.default_rng(seed)
    for n in [1, 2, 3, 10, 63, 500]:
        edges = np.sort(rng.uniform(-20, 20, n + 1))
        edges = np.unique(edges)
        if len(edges) < 2:
            continue
        el = [float(e) for e in edges]
        nb = len(el) - 1
        for x in _variable_probe_points(el, rng):
            x = float(x)
            got = oracle.find_bin_variable(el, x)
            if math.isnan(x):
                exp = nb + 1
            else:
                exp = bisect.bisect_right(el, x)
            assert got == exp, f"edges n={nb} x={x!r}: {got} != bisect {exp}"
            if not math.isnan(x):
                scan = 0 if x < el[0] else nb + 1
                for j in range(nb):
                    if el[j] <= x < el[j + 1]:
                        scan = j + 1
                assert got == scan, f"edges n={nb} x={x!r}: {got} != scan {scan}"


def check_variable_matches_fixed_on_dyadic_edges():
    """With the edges of the dyadic fixed axis, both searches agree wherever
    the formula's subtraction x - min is exact (then every step is exact, so
    both sides implement the same lower-inclusive bins)."""
    edges = [-4 + 0.5 * k for k in range(17)]
    rng = np.random.default_rng(5)
    pts = _variable_probe_points(edges, rng)
    checked = 0
    for x in pts:
        x = float(x)
        if math.isfinite(x) and Fraction(x) + 4 != Fraction(x + 4.0):
            continue
        checked += 1
        assert oracle.find_bin_variable(edges, x) == oracle.find_bin_fixed(16, -4.0, 4.0, x), x
    assert checked > 300


def check_nd_enumerated():
    """Every bin of a 4 x 5 x 6 (with flows) 3D histogram, and of a 2D one,
    gets exactly the point placed in it, x fastest."""
    axes = [oracle_axis_fixed(2, 0.0, 2.0), oracle_axis_fixed(3, 0.0, 3.0),
            oracle_axis_fixed(4, 0.0, 4.0)]

    def coord(b, n):
        if b == 0:
            return -0.5
        if b == n + 1:
            return n + 0.5
        return b - 0.5

    pts, exp = [], []
    for bz in range(6):
        for by in range(5):
            for bx in range(4):
                pts.append((coord(bx, 2), coord(by, 3), coord(bz, 4)))
                exp.append(bx + 4 * (by + 5 * bz))
    v = np.array(pts).T.copy()
    got = oracle.locate(axes, v)
    assert list(got) == exp, "3D linearisation"
    assert sorted(exp) == list(range(120))
    v2 = v[:2].copy()
    got2 = oracle.locate(axes[:2], v2)
    exp2 = [p % 20 for p in exp]
    assert list(got2) == exp2, "2D linearisation"


def oracle_axis_fixed(n, a, b):
    return {"kind": "fixed", "nbins": n, "xmin": a, "xmax": b}


# --------------------------------------------------------------- fill ------


def check_golden_fill():
    for case in golden_io.fill_cases():
        axes = [ax if ax["kind"] == "fixed" else {"kind": "variable", "edges": ax["edges"]}
                for ax in case["axes"]]
        v = np.array(case["events"], dtype=np.float64).T.copy()
        w = np.array(case["weights"], dtype=np.float64)
        r = oracle.fill(axes, v, w, stat_overflows=bool(case["stat_overflows"]))
        nb = oracle.nbins_total(axes)
        exp_bins = np.zeros(nb)
        for k, val in case["bins"].items():
            exp_bins[k] = val
        for arr in (r.bins_seq, r.bins_acc):
            assert np.array_equal(arr, exp_bins), f"{case['name']}: bins {arr} != {exp_bins}"
        for arr in (r.stats_seq, r.stats_acc):
            assert list(arr) == case["stats"], f"{case['name']}: stats {list(arr)} != {case['stats']}"


def _terms_numpy(v, w):
    """Statistic terms, each rounded once, computed with numpy's elementwise
    binary64 operations (w*x*x evaluated as (w*x)*x)."""
    ndim = v.shape[0]
    x = v[0]
    wx = w * x
    t = [w, w * w, wx, wx * x]
    if ndim >= 2:
        y = v[1]
        wy = w * y
        t += [wy, wy * y, wx * y]
    if ndim >= 3:
        z = v[2]
        wy = w * v[1]
        wz = w * z
        t += [wz, wz * z, wx * z, wy * z]
    return t


def _in_range_mask(axes, v):
    m = np.ones(v.shape[1], dtype=bool)
    for d, ax in enumerate(axes):
        if ax["kind"] == "fixed":
            m &= (v[d] >= ax["xmin"]) & (v[d] < ax["xmax"])
        else:
            e = np.asarray(ax["edges"])
            m &= (v[d] >= e[0]) & (v[d] < e[-1])
    return m


def check_fill_counts_vs_numpy(seed=6):
    """Counts against numpy.histogram (in-range bins, lower-inclusive) and the
    flow bins against direct comparisons; unit weights total N."""
    rng = np.random.default_rng(seed)
    n = 20000
    # variable axis
    edges = np.unique(np.sort(rng.uniform(-3, 3, 41)))
    x = rng.normal(0, 1.5, n)
    r = oracle.fill([{"kind": "variable", "edges": edges}], x.reshape(1, n))
    h, _ = np.histogram(x[(x >= edges[0]) & (x < edges[-1])], bins=edges)
    assert np.array_equal(r.counts[1:-1], h.astype(np.uint64))
    assert r.counts[0] == np.count_nonzero(x < edges[0])
    assert r.counts[-1] == np.count_nonzero(x >= edges[-1])
    assert int(r.counts.sum()) == n
    # unit weights: Sum w over in-range = in-range count = Sum w^2
    inr = int(r.counts[1:-1].sum())
    assert r.stats_acc[0] == n and r.stats_acc[1] == inr and r.stats_acc[2] == inr
    # fixed axis, dyadic, against numpy.histogram on the equivalent edges
    x = rng.uniform(-5, 5, n)
    r = oracle.fill([oracle_axis_fixed(16, -4.0, 4.0)], x.reshape(1, n))
    e = np.array([-4 + 0.5 * k for k in range(17)])
    h, _ = np.histogram(x[(x >= -4) & (x < 4)], bins=e)
    assert np.array_equal(r.counts[1:-1], h.astype(np.uint64))
    assert r.counts[0] == np.count_nonzero(x < -4) and r.counts[-1] == np.count_nonzero(x >= 4)


def check_fill_sums_vs_library(seed=7):
    """Per-bin weighted sums: the event-order sum against numpy.bincount (a
    sequential C loop) bit for bit, the compensated sum against math.fsum."""
    rng = np.random.default_rng(seed)
    n = 20000
    axes = [oracle_axis_fixed(50, -2.0, 2.0)]
    x = rng.normal(0, 1, n)
    w = rng.uniform(-1, 3, n)
    r = oracle.fill(axes, x.reshape(1, n), w)
    b = oracle.locate(axes, x.reshape(1, n))
    nb = 52
    seq = np.bincount(b, weights=w, minlength=nb)
    assert np.array_equal(r.bins_seq, seq)
    assert np.array_equal(r.counts, np.bincount(b, minlength=nb).astype(np.uint64))
    for g in range(nb):
        ref = math.fsum(w[b == g])
        assert abs(r.bins_acc[g] - ref) <= 2 * math.ulp(ref) + 1e-300, g
        assert abs(r.bins_abs[g] - math.fsum(np.abs(w[b == g]))) <= 1e-12 * r.bins_abs[g] + 1e-300


def check_stats_vs_fsum(seed=8):
    """Statistics: compensated sums against math.fsum of the rounded terms,
    event-order sums against numpy.cumsum (sequential), over in-range events."""
    rng = np.random.default_rng(seed)
    n = 20000
    cases = [
        [oracle_axis_fixed(40, -2.0, 2.0)],
        [oracle_axis_fixed(30, -2.0, 2.0), {"kind": "variable", "edges": np.linspace(-1.5, 3.0, 21)}],
        [oracle_axis_fixed(10, -2.0, 2.0), oracle_axis_fixed(11, -1.0, 3.0), oracle_axis_fixed(12, -2.5, 1.5)],
    ]
    for axes in cases:
        ndim = len(axes)
        v = np.empty((ndim, n))
        v[0] = rng.normal(0, 1, n)
        if ndim >= 2:
            v[1] = rng.normal(0.7, 1.1, n)
        if ndim >= 3:
            v[2] = rng.normal(-0.4, 0.9, n)
        w = rng.uniform(-0.5, 2.0, n)
        r = oracle.fill(axes, v, w)
        m = _in_range_mask(axes, v)
        terms = _terms_numpy(v[:, m], w[m])
        assert r.stats_acc[0] == n and r.stats_seq[0] == n
        for k, t in enumerate(terms, start=1):
            ref = math.fsum(t)
            assert abs(r.stats_acc[k] - ref) <= 4 * math.ulp(ref) + 1e-300, (ndim, k)
            assert r.stats_seq[k] == np.cumsum(t)[-1], (ndim, k)


def check_stats_closed_form_centres():
    """Unit weights at every bin centre of [0, 1) with 10 bins, then weight k
    in bin k: Sum w, Sum w^2, Sum wx, Sum wx^2 against exact rational sums of
    the same doubles."""
    cs = [float(Fraction(2 * k - 1, 20)) for k in range(1, 11)]
    for ws in ([1.0] * 10, [float(k) for k in range(1, 11)]):
        r = oracle.fill([oracle_axis_fixed(10, 0.0, 1.0)], np.array([cs]), np.array(ws))
        F = [Fraction(c) for c in cs]
        W = [Fraction(w) for w in ws]
        exact = [sum(W), sum(w * w for w in W), sum(w * c for w, c in zip(W, F)),
                 sum(w * c * c for w, c in zip(W, F))]
        for k, e in enumerate(exact, start=1):
            assert abs(Fraction(r.stats_acc[k]) - e) <= Fraction(1, 2 ** 48) * abs(e), k
        assert list(r.counts) == [0] + [1] * 10 + [0]


def check_flows_and_specials():
    """NaN coordinates go to overflow and stay out of the statistics; a NaN
    or infinite weight propagates into its bin; stat_overflows switches the
    flow entries into the statistics."""
    axes = [oracle_axis_fixed(4, 0.0, 1.0)]
    v = np.array([[0.1, NAN, 2.0, -1.0, 0.75]])
    w = np.array([1.0, 5.0, 7.0, 11.0, 2.0])
    r = oracle.fill(axes, v, w)
    assert list(r.counts) == [1, 1, 0, 0, 1, 2]
    assert r.bins_acc[5] == 12.0 and r.bins_acc[0] == 11.0
    assert r.stats_acc[0] == 5 and r.stats_acc[1] == 3.0
    r2 = oracle.fill(axes, np.array([[2.0, -1.0, 0.75]]), np.array([7.0, 11.0, 2.0]),
                     stat_overflows=True)
    assert r2.stats_acc[1] == 20.0 and r2.stats_acc[3] == 4.5
    r3 = oracle.fill(axes, np.array([[0.1, 0.15, 0.9]]), np.array([NAN, 1.0, INF]))
    assert math.isnan(r3.bins_acc[1]) and math.isnan(r3.bins_seq[1])
    assert r3.bins_acc[4] == INF and r3.bins_seq[4] == INF


def check_fills_accumulate(seed=9):
    """Two fills equal one fill over the concatenation (the running sums of
    the previous bulk are combined, never overwritten)."""
    rng = np.random.default_rng(seed)
    axes = [oracle_axis_fixed(20, -2.0, 2.0)]
    x = rng.normal(0, 1, 5000).reshape(1, -1)
    w = rng.uniform(0, 1, 5000)
    acc = oracle.Accumulator(axes)
    acc.fill(x[:, :2000], w[:2000])
    acc.fill(x[:, 2000:], w[2000:])
    a = acc.result()
    b = oracle.fill(axes, x, w)
    assert np.array_equal(a.counts, b.counts)
    assert np.array_equal(a.bins_seq, b.bins_seq)
    assert np.array_equal(a.stats_seq, b.stats_seq)


def check_sumw2_vs_bincount(seed=10):
    """Per-bin sum of squared weights against numpy.bincount of w*w over the
    oracle's own (pinned) bins, and math.fsum per bin; unit weights give the
    counts."""
    rng = np.random.default_rng(seed)
    axes = [oracle_axis_fixed(20, -1.0, 1.0)]
    x = rng.normal(0, 0.7, 5000)
    w = rng.uniform(-2.0, 3.0, 5000)
    s2, a2 = oracle.sumw2(axes, x.reshape(1, -1), w)
    g = oracle.locate(axes, x.reshape(1, -1))
    ref = np.bincount(g, weights=w * w, minlength=22)
    assert np.allclose(s2, ref, rtol=1e-13, atol=0.0)
    for k in range(22):
        assert s2[k] == math.fsum((w * w)[g == k])
        assert a2[k] == math.fsum(np.abs(w * w)[g == k]) or np.isclose(a2[k], np.sum(np.abs(w * w)[g == k]))
    c, _ = oracle.sumw2(axes, x.reshape(1, -1), None)
    assert np.array_equal(c, np.bincount(g, minlength=22).astype(np.float64))


def check_define_filter_vs_python_loops(seed=11):
    """The Filter/Define restatement against per-event Python float
    arithmetic (IEEE binary64, one rounding per operation) on small inputs,
    with zeros, NaN, infinities and signed zeros in the columns."""
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 2, 300)
    y = rng.normal(0, 2, 300)
    x[::7] = 0.0
    x[1::11] = -0.0
    y[2::13] = math.nan
    x[3::17] = math.inf
    defines = [(oracle.DEF_SUMSQ, 0, 1), (oracle.DEF_HYPOT, 0, 1), (oracle.DEF_MUL, 0, 1),
               (oracle.DEF_ADD, 0, 1), (oracle.DEF_SUB, 0, 1), (oracle.DEF_COL, 1, 0)]
    filters = [(0, oracle.FLT_NE, 0.0), (1, oracle.FLT_LT, 3.0)]
    mask, vals = oracle.define_filter([x, y], defines, filters)
    for i in range(300):
        a, b = float(x[i]), float(y[i])
        assert mask[i] == ((a != 0.0) and (b < 3.0))
        aa, bb = a * a, b * b
        s2 = aa + bb
        want = [s2, math.sqrt(s2) if s2 >= 0 or math.isnan(s2) else math.nan, a * b, a + b, a - b, b]
        for k, wv in enumerate(want):
            got = float(vals[k][i])
            assert (math.isnan(got) and math.isnan(wv)) or got == wv, (i, k, got, wv)
    for op, fn in [(oracle.FLT_EQ, lambda a: a == 1.5), (oracle.FLT_LE, lambda a: a <= 1.5),
                   (oracle.FLT_GT, lambda a: a > 1.5), (oracle.FLT_GE, lambda a: a >= 1.5)]:
        m, _ = oracle.define_filter([x], [(oracle.DEF_COL, 0, 0)], [(0, op, 1.5)])
        assert all(m[i] == fn(float(x[i])) for i in range(300))


def check_exact_stats_vs_fractions(seed=12):
    """The exact statistics against exact rational sums of the same rounded
    terms (fractions.Fraction), rounded once by float(); specials."""
    rng = np.random.default_rng(seed)
    axes = [oracle_axis_fixed(10, -2.0, 2.0)]
    x = rng.normal(0, 1.2, 400)
    w = rng.uniform(-3, 3, 400) * 10.0 ** rng.integers(-12, 12, 400)
    got = oracle.exact_stats(axes, x, w)
    g = oracle.locate(axes, x.reshape(1, -1))
    m = (g >= 1) & (g <= 10)
    xs, ws = x[m].tolist(), w[m].tolist()
    terms = [ws, [a * a for a in ws], [a * b for a, b in zip(ws, xs)], [(a * b) * b for a, b in zip(ws, xs)]]
    for k in range(4):
        want = float(sum(Fraction(t) for t in terms[k]))
        assert got[k] == want, (k, got[k], want)
    w2 = w.copy()
    w2[int(np.flatnonzero(m)[0])] = math.nan
    assert all(math.isnan(v) for v in oracle.exact_stats(axes, x, w2))
    w3 = w.copy()
    w3[int(np.flatnonzero(m)[1])] = math.inf
    assert oracle.exact_stats(axes, x, w3)[0] == math.inf
    # 2D and 3D: ROOT's TH2/TH3 term sets (R6), an entry taken only when
    # every axis is in range, per-event terms from Python float arithmetic
    for ndim in (2, 3):
        axs = [oracle_axis_fixed(10, -2.0, 2.0), {"kind": "variable", "edges": np.array([-1.0, 0.0, 0.5, 3.0])},
               oracle_axis_fixed(7, -1.5, 2.5)][:ndim]
        v = np.stack([rng.normal(0, 1.2, 300), rng.normal(0.5, 1.0, 300), rng.normal(0.2, 1.3, 300)][:ndim])
        w = rng.uniform(-3, 3, 300) * 10.0 ** rng.integers(-9, 9, 300)
        got = oracle.exact_stats(axs, v, w)
        lo = [-2.0, -1.0, -1.5]
        hi = [2.0, 3.0, 2.5]
        sel = [i for i in range(300) if all(lo[d] <= v[d, i] < hi[d] for d in range(ndim))]
        assert 50 < len(sel) < 300
        rows = []
        for i in sel:
            wi, xi = float(w[i]), float(v[0, i])
            wxi = wi * xi
            r = [wi, wi * wi, wxi, wxi * xi]
            if ndim >= 2:
                yi = float(v[1, i])
                wyi = wi * yi
                r += [wyi, wyi * yi, wxi * yi]
            if ndim >= 3:
                zi = float(v[2, i])
                wzi = wi * zi
                r += [wzi, wzi * zi, wxi * zi, wyi * zi]
            rows.append(r)
        nterm = {2: 7, 3: 11}[ndim]
        assert len(got) == nterm
        for k in range(nterm):
            want = float(sum(Fraction(r[k]) for r in rows))
            assert got[k] == want, (ndim, k, got[k], want)


def check_chunk_parallel_fill_and_locate(seed=13):
    """The chunk-parallel modes (oracle_fill_mt, oracle_locate_mt) that the
    full-size parity tests use as their reference, at several thread counts
    (more threads than events included) and ragged sizes: bins from
    numpy.searchsorted (variable axis) and exact dyadic arithmetic (fixed
    axis), counts from numpy.bincount of those bins, compensated per-bin and
    statistics sums within a few ulps of math.fsum, every event counted once.
    A hand-made bin whose compensated value exists only in the correction
    terms (1e16 + 1 - 1e16 inside each chunk) pins the merge of those terms."""
    rng = np.random.default_rng(seed)
    edges = np.unique(np.sort(rng.uniform(-3, 3, 37)))
    assert len(edges) == 37  # 36 bins + 2 flows: linear stride 38
    ax_var = {"kind": "variable", "edges": edges}
    ax_fix = oracle_axis_fixed(16, -4.0, 4.0)

    def bins_var(x):
        return np.searchsorted(edges, x, side="right")  # NaN sorts last: overflow

    def bins_fix(x):
        b = np.where(x < -4.0, 0, np.where(x >= 4.0, 17, 0))
        inr = (x >= -4.0) & (x < 4.0)
        b[inr] = 1 + np.floor(2.0 * (x[inr] + 4.0)).astype(np.int64)  # exact for x = k 2^-20
        return b

    for n in (0, 1, 5, 7, 1001, 20011):
        x = rng.normal(0, 1.6, n)
        x[::97] = NAN
        y = rng.integers(-5 * 2 ** 20, 5 * 2 ** 20, n) * 2.0 ** -20
        w = rng.uniform(-0.5, 2.0, n)
        for axes, v, gi in (([ax_var], x.reshape(1, n), bins_var(x)),
                            ([ax_var, ax_fix], np.stack([x, y]), bins_var(x) + 38 * bins_fix(y))):
            nb = oracle.nbins_total(axes)
            inr = np.ones(n, dtype=bool)
            for d, ax in enumerate(axes):
                bd = bins_var(v[d]) if ax["kind"] == "variable" else bins_fix(v[d])
                inr &= (bd >= 1) & (bd <= (len(edges) - 1 if ax["kind"] == "variable" else 16))
            terms = _terms_numpy(v[:, inr], w[inr])
            for threads in (2, 3, 7, 16):
                got = oracle.locate(axes, v, threads=threads)
                assert np.array_equal(got, gi), f"locate_mt n={n} threads={threads}"
                r = oracle.fill(axes, v, w, threads=threads)
                assert np.array_equal(r.counts, np.bincount(gi, minlength=nb).astype(np.uint64)), \
                    f"fill_mt counts n={n} threads={threads}"
                assert r.stats_acc[0] == n and r.stats_seq[0] == n
                for g in np.flatnonzero(r.counts):
                    ref = math.fsum(w[gi == g])
                    assert abs(r.bins_acc[g] - ref) <= 2 * math.ulp(ref) + 1e-300, (n, threads, g)
                    assert abs(r.bins_seq[g] - ref) <= 1e-12 * r.bins_abs[g] + 1e-300, (n, threads, g)
                for k, t in enumerate(terms, start=1):
                    ref = math.fsum(t)
                    assert abs(r.stats_acc[k] - ref) <= 4 * math.ulp(ref) + 1e-300, (n, threads, k)
    # every chunk holds 1e16, 1, -1e16 in bin 1: its value lives in the
    # compensation term, which the merge must carry over
    n = 12
    x = np.full(n, float(edges[0]))
    w = np.tile([1e16, 1.0, -1e16], 4)
    for threads in (2, 4):
        r = oracle.fill([ax_var], x.reshape(1, n), w, threads=threads)
        assert r.bins_acc[1] == 4.0, (threads, r.bins_acc[1])
        r = oracle.fill([ax_var], x.reshape(1, n), w * 0.5, threads=threads)
        assert r.stats_acc[1] == 2.0, (threads, r.stats_acc[1])


ALL_CHECKS = [
    check_golden_fixed, check_golden_variable, check_fixed_dyadic_exact,
    check_fixed_vs_rational, check_fixed_centres, check_fixed_range_edges,
    check_fixed_monotone, check_variable_vs_bisect_and_scan,
    check_variable_matches_fixed_on_dyadic_edges, check_nd_enumerated,
    check_golden_fill, check_fill_counts_vs_numpy, check_fill_sums_vs_library,
    check_stats_vs_fsum, check_stats_closed_form_centres, check_flows_and_specials,
    check_fills_accumulate, check_sumw2_vs_bincount, check_define_filter_vs_python_loops,
    check_exact_stats_vs_fractions, check_chunk_parallel_fill_and_locate,
]
