"""Test helpers: key <-> double conversion written independently of the
library, tolerance checks, and GPU fill runners (through the C ABI)."""
from __future__ import annotations

import math
import struct

import numpy as np

INT64_MIN = -(1 << 63)
INT64_MAX = (1 << 63) - 1


def double_of_key(k: int) -> float:
    """Inverse of the library's ordered key (-0 shares key 0 with +0)."""
    b = k if k >= 0 else ((-k) | (1 << 63))
    return struct.unpack("<d", struct.pack("<Q", b & ((1 << 64) - 1)))[0]


def key_of_double(x: float) -> int:
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    mag = b & ((1 << 63) - 1)
    if mag > 0x7FF0000000000000:
        return INT64_MAX - 1
    return -mag if b >> 63 else mag


def assert_sums_close(got, ref, scale, rtol, what, atol=0.0):
    """|got - ref| <= rtol * scale + atol elementwise, with equal non-finite
    values (inf == inf, nan == nan) accepted."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    both_nan = np.isnan(got) & np.isnan(ref)
    same_inf = np.isinf(got) & np.isinf(ref) & (np.sign(got) == np.sign(ref))
    with np.errstate(invalid="ignore"):
        err = np.abs(got - ref)
        lim = rtol * scale + atol
        bad = ~(both_nan | same_inf) & ~(err <= lim)
    if np.any(bad):
        i = int(np.flatnonzero(bad)[0])
        raise AssertionError(f"{what}: {int(bad.sum())} entries out of tolerance; first at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r} err {err[i]:.3e} lim {lim[i]:.3e}")
    with np.errstate(invalid="ignore", divide="ignore"):
        rel = np.where(scale > 0, err / np.where(scale > 0, scale, 1.0), 0.0)
    rel = rel[~(both_nan | same_inf)]
    return float(rel.max()) if rel.size else 0.0


def to_device(a):
    import torch
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    return a


def gpu_fill(axes, values, weights=None, flags=0, chunks=1):
    """Book, fill (optionally in several slices), return (bins, stats, counts|None)."""
    import torch
    from paper_2401_13310_gb300 import binding as B
    v = np.ascontiguousarray(values, dtype=np.float64)
    if v.ndim == 1:
        v = v.reshape(1, -1)
    n = v.shape[1]
    h = B.Hist(axes, flags)
    try:
        bounds = [n * i // chunks for i in range(chunks + 1)]
        for a, b in zip(bounds, bounds[1:]):
            vd = to_device(np.ascontiguousarray(v[:, a:b]))
            wd = to_device(None if weights is None else np.ascontiguousarray(weights[a:b]))
            h.fill(vd, wd)
            torch.cuda.synchronize()
        bins, stats = h.result()
        counts = None
        if weights is None or (flags & B.HIST_TRACK_COUNTS):
            counts = h.counts()
        return bins, stats, counts
    finally:
        h.close()


def check_against_oracle(axes, values, weights, bins, stats, counts, ref, rtol_bins=1e-12,
                         rtol_stats=1e-12, what=""):
    """Counts bit-exact; unit-weight bins exact; weighted bins and statistics
    within rtol of the compensated oracle sums, relative to sum |term|."""
    if counts is not None:
        assert np.array_equal(counts, ref.counts), f"{what}: counts differ at " \
            f"{np.flatnonzero(counts != ref.counts)[:10]}"
    if weights is None:
        assert np.array_equal(bins, ref.counts.astype(np.float64)), f"{what}: unit-weight bins differ"
    else:
        assert_sums_close(bins, ref.bins_acc, ref.bins_abs, rtol_bins, f"{what} bins")
    assert stats[0] == ref.stats_acc[0], f"{what}: entry count {stats[0]} != {ref.stats_acc[0]}"
    return assert_sums_close(stats[1:], ref.stats_acc[1:], ref.stats_abs[1:], rtol_stats, f"{what} stats")


def edge_probe_values(axis, thresholds, rng, nrand=2000):
    """Coordinates that stress find-bin: every threshold and its predecessor
    key, signed zeros, infinities, NaNs, subnormals, huge values, random."""
    pts = []
    for k in range(1, len(thresholds) - 1):
        t = int(thresholds[k])
        for dk in (-2, -1, 0, 1):
            kk = t + dk
            if -0x7FF0000000000000 <= kk <= 0x7FF0000000000000:
                pts.append(double_of_key(kk))
    pts += [0.0, -0.0, math.inf, -math.inf, math.nan, -math.nan, 5e-324, -5e-324, 1e-310,
            1e308, -1e308, 1e30, -1e30, 3.4e38, -3.4e38, 1e-30, -1e-30]
    if axis["kind"] == "fixed":
        lo, hi = axis["xmin"], axis["xmax"]
    else:
        lo, hi = float(axis["edges"][0]), float(axis["edges"][-1])
    span = hi - lo
    pts += list(rng.uniform(lo - 0.1 * span, hi + 0.1 * span, nrand))
    return np.array(pts, dtype=np.float64)
