"""The FP32 estimate that locates fixed axes, emulated on the CPU.

For a fixed axis the kernels evaluate v = fmaf(x24, scale, offset) on the
coordinate truncated to 24 significant bits, take t = fadd_rd(v, 1.5 2^23)
so that the bits of t hold floor(v), and trust that bin (clamped to the flow
bins) when the fraction of v is more than eps from an integer.  The library
computes scale, offset and eps on the host (hist_axis_affine); this file
replays the device's single-precision operations exactly (the fused
multiply-add and the round-down addition by rational arithmetic, the rest by
numpy float32, whose operations round to nearest) and checks, over many
axes and over coordinates at every kind of boundary, that every trusted
estimate is the Sec. 3.1 bin of the oracle.  A second test shows that the
check has teeth: with eps = 0 the same replay trusts wrong bins.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import binding as B
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import double_of_key

MAGIC = 12582912.0  # 1.5 * 2^23
TWO128 = Fraction(2) ** 128


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2401_13310_gb300 import _build
    _build.build()
    B.load()
    oracle.build()


def _f32(r: Fraction, down: bool) -> float:
    """r rounded to binary32: to nearest-even, or toward -inf; +-inf when
    the rounded magnitude reaches 2^128 (round-down keeps the largest finite
    value for a positive r)."""
    if r == 0:
        return 0.0
    neg = r < 0
    a = -r if neg else r
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    q = max(e, -126) - 23  # the quantum of the binade (subnormals share 2^-149)
    m = a / Fraction(2) ** q
    fl = m.numerator // m.denominator
    rem = m - fl
    if down:
        mi = fl + (1 if (neg and rem > 0) else 0)
    else:
        mi = fl + (1 if (rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1)) else 0)
    v = Fraction(mi) * Fraction(2) ** q
    if v >= TWO128:
        if down and not neg:
            return float(np.finfo(np.float32).max)
        return -math.inf if neg else math.inf
    return -float(v) if neg else float(v)


def _bits64(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _bits32(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _device_estimate(x: float, scale: float, offset: float, eps: float, nbins: int):
    """(trusted, bin) as the kernels form them for coordinate x."""
    b = _bits64(x)
    ef = (b >> 52) & 0x7FF
    if not (897 <= ef < 1151):  # |x| outside [2^-126, 2^128): thresholds only
        return False, None
    x24 = struct.unpack("<d", struct.pack("<Q", b & ~((1 << 29) - 1)))[0]
    v = _f32(Fraction(x24) * Fraction(scale) + Fraction(offset), down=False)
    if math.isinf(v):
        t = v
    else:
        t = _f32(Fraction(v) + Fraction(MAGIC), down=True)
    k = (_bits32(t) - 0x4B400000) & 0xFFFFFFFF
    k = k - (1 << 32) if k >= (1 << 31) else k
    with np.errstate(invalid="ignore", over="ignore"):
        f32 = np.float32
        fr = f32(v) - (f32(t) - f32(MAGIC))
        sure = bool(np.abs(fr - f32(0.5)) < (f32(0.5) - f32(eps)))
    return sure, min(max(k, 0), nbins + 1)


def _axes():
    out = [W.fixed(1000, -5.0, 5.0), W.fixed(100, 0.0, 1.0), W.fixed(1000, 0.0, 1.0), W.fixed(7, -0.3, 0.4),
           W.fixed(1, 2.0, 3.0), W.fixed(100000, 0.0, 300.0), W.fixed(3163, -math.pi, math.pi),
           W.fixed(1022, -3.0, 3.0), W.fixed(1000, 1e6, 1e6 + 1.0), W.fixed(300, -1e-6, 3e-6),
           W.fixed((1 << 21) - 1, 0.0, 1.0), W.fixed(10, 1e30, 3e30), W.fixed(64, -2.0 ** 20, 2.0 ** 20)]
    rng = np.random.default_rng(31)
    for _ in range(40):
        nbins = int(10 ** rng.uniform(0, math.log10(2e6)))
        width = 10 ** rng.uniform(-6, 6)
        xmin = float(rng.choice([-1, 1]) * 10 ** rng.uniform(-6, 6) * rng.uniform(0, 1))
        out.append(W.fixed(max(nbins, 1), xmin, xmin + width))
    return out


def _points(axis, T, rng, nthr=150, nrand=150):
    nb, lo, hi = axis["nbins"], axis["xmin"], axis["xmax"]
    w = hi - lo
    ks = np.arange(1, nb + 2)
    if ks.size > nthr:
        ks = np.concatenate([ks[:5], ks[-5:], rng.choice(ks, nthr - 10, replace=False)])
    pts = []
    for k in ks:
        for d in (-2, -1, 0, 1, 2):
            key = int(T[k]) + d
            if -0x7FF0000000000000 <= key <= 0x7FF0000000000000:
                pts.append(double_of_key(key))
    pts += list(rng.uniform(lo - w / 4, hi + w / 4, nrand))
    pts += [lo + w * (i + 0.5) / nb for i in rng.integers(0, nb, 20)]  # bin centres
    pts += [0.0, -0.0, 1e-30, -1e-30, 2.0 ** -126, -(2.0 ** -126), 1e30, -1e30, 3e38, -3e38, 1e300, -1e300,
            math.inf, -math.inf, math.nan]
    return pts


def _replay(eps_override=None):
    """Replays every point of every axis that takes the estimate; returns
    the number of points checked, of trusted estimates that are wrong, and
    per axis (eps, fraction of uniform in-range points trusted)."""
    rng = np.random.default_rng(32)
    checked = wrong = 0
    used = []
    for axis in _axes():
        est = B.hist_axis_affine(axis)
        if est is None:
            continue
        scale, offset, eps = est
        if eps_override is not None:
            eps = eps_override
        T = B.hist_axis_thresholds(axis)
        nb, lo, hi = axis["nbins"], axis["xmin"], axis["xmax"]
        for x in _points(axis, T, rng):
            sure, k = _device_estimate(x, scale, offset, eps, nb)
            checked += 1
            if sure and k != oracle.find_bin_fixed(nb, lo, hi, x):
                wrong += 1
        inside = rng.uniform(lo, hi, 300)
        frac = sum(_device_estimate(float(x), scale, offset, eps, nb)[0] for x in inside) / inside.size
        used.append((eps, frac))
    return checked, wrong, used


def test_trusted_estimates_are_the_exact_bins():
    checked, wrong, used = _replay()
    assert wrong == 0, (wrong, checked)
    assert len(used) >= 30
    # the bound is not vacuous: a uniform in-range coordinate is decided by
    # the estimate unless v lands within eps of an integer (probability about
    # 2 eps; 0.08 is three standard deviations of 300 samples)
    for eps, frac in used:
        assert frac >= 1.0 - 2.0 * eps - 0.08, (eps, frac)


def test_without_the_bound_the_estimate_is_wrong_somewhere():
    checked, wrong, _ = _replay(eps_override=0.0)
    assert wrong > 0, checked
