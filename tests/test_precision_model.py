"""Sensitivity of the reduced-precision bound checks, on a CPU model.

The GPU tests hold the FP32 compensated bins (HIST_PREC_FP32C) and the
compensated per-bin sums of w^2 (HIST_SUMW2) to 1e-12 of the bin's sum of
|terms|.  This file models the same FP32 arithmetic on the CPU (numpy
float32 scalars, one rounding per operation) and shows both sides of that
check: the arithmetic as written stays inside the tolerance (and inside its
stated per-block worst-case bound), while the same arithmetic with the TwoSum error
term dropped -- the plausible mistake -- lands far outside it.  Nothing here
touches the GPU or the oracle; math.fsum gives the exact reference sums.
"""
import math
import struct

import numpy as np

RTOL = 1e-12
f32 = np.float32


def split(w: float):
    """w = hi + lo: hi = w's leading 24 significant bits (truncated), lo =
    the remainder rounded to FP32 (|w - hi - lo| <= 2^-48 |w|)."""
    b = struct.unpack("<Q", struct.pack("<d", w))[0]
    hi = struct.unpack("<d", struct.pack("<Q", b & ~((1 << 29) - 1)))[0]
    return f32(hi), f32(w - hi)


def two_sum_into(S, C, a, lo, drop_err=False):
    """S <- fl(S + a) with the rounding error recovered exactly (Knuth's
    TwoSum on the old value) and added, with lo, to the compensation word C."""
    old = S
    s = f32(old + a)
    bv = f32(s - old)
    err = f32(f32(old - f32(s - bv)) + f32(a - bv))
    C = f32(C + (lo if drop_err else f32(err + lo)))
    return s, C


def model_fp32c(blocks, drop_err=False):
    total = 0.0
    for ws in blocks:
        S, C = f32(0), f32(0)
        for w in ws:
            hi, lo = split(w)
            S, C = two_sum_into(S, C, hi, lo, drop_err)
        total = total + (float(S) + float(C))  # flush: binary64 sum of the two words, blocks in order
    return total


def model_sumw2(blocks, drop_err=False):
    total = 0.0
    for ws in blocks:
        S, C = f32(0), f32(0)
        for w in ws:
            hi, lo = split(w)
            ph = f32(float(hi) * float(hi))
            pe = f32(float(hi) * float(hi) - float(ph))          # exact: hi*hi has 48 bits
            pl = f32(2.0 * float(hi) * float(lo) + float(pe))
            S, C = two_sum_into(S, C, ph, pl, drop_err)
        total = total + (float(S) + float(C))
    return total


def _blocks(seed, nblocks=600, per_block=16):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.5, 1.5, per_block).tolist() for _ in range(nblocks)]


def test_fp32c_model_inside_tolerance_and_dropped_error_outside():
    blocks = _blocks(1)
    allw = [w for ws in blocks for w in ws]
    exact = math.fsum(allw)
    A = math.fsum(abs(w) for w in allw)
    m, nb = 16, len(blocks)
    stated = 2.0 ** -48 * ((m + 1) ** 2 + 1) * A + nb * 2.0 ** -53 * A
    good = abs(model_fp32c(blocks) - exact)
    bad = abs(model_fp32c(blocks, drop_err=True) - exact)
    assert good <= stated and good <= RTOL * A, (good, stated)
    assert bad > RTOL * A, f"a dropped TwoSum error term would pass the check: {bad / A:.3g}"


def test_sumw2_model_inside_tolerance_and_dropped_error_outside():
    blocks = _blocks(2)
    allw2 = [w * w for ws in blocks for w in ws]
    exact = math.fsum(allw2)
    A = exact
    m, nb = 16, len(blocks)
    stated = 2.0 ** -44 * A + 2.0 ** -48 * ((m + 1) ** 2 + 1) * A + nb * 2.0 ** -53 * A
    good = abs(model_sumw2(blocks) - exact)
    bad = abs(model_sumw2(blocks, drop_err=True) - exact)
    assert good <= stated and good <= RTOL * A, (good, stated)
    assert bad > RTOL * A, f"a dropped TwoSum error term would pass the check: {bad / A:.3g}"


def test_split_is_exact_to_48_bits():
    rng = np.random.default_rng(3)
    for w in rng.uniform(-300, 300, 2000):
        hi, lo = split(float(w))
        assert abs(float(w) - float(hi) - float(lo)) <= 2.0 ** -48 * abs(w)
