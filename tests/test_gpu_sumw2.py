"""Per-bin sum of squared weights (HIST_SUMW2, ROOT's Sumw2) against the
oracle, in every precision mode, for shared-memory bins (compensated FP32
words) and global bins (binary64 atomics), unit and weighted fills mixed.
Every bin within 1e-12 of A = the sum of w^2 over its entries (the tolerance
of the binary64 paths).  The stated bound of the compensated FP32 words, with
m = the bin's entries in one block and B blocks,
    |err| <= 2^-44 A + 2^-48 ((m + 1)^2 + 1) A + B 2^-53 A,
is a worst case; the errors measured are near 1e-14 A, and a dropped TwoSum
error term would be orders of magnitude above the tolerance
(tests/test_precision_model.py)."""
import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import assert_sums_close, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


RTOL = 1e-12


@pytest.mark.parametrize("name,n", [("2a", 1_000_003), ("2b", 1_000_003), ("3a", 300_001), ("3b", 500_001)])
@pytest.mark.parametrize("prec", ["fp64", "fp32c", "f64atomic"])
def test_sumw2_matches_oracle(B, name, n, prec):
    import torch
    wl = W.CONFIGS[name](n=n)
    flags = B.HIST_SUMW2 | {"fp64": B.HIST_PREC_FP64, "fp32c": B.HIST_PREC_FP32C,
                            "f64atomic": B.HIST_PREC_F64ATOMIC}[prec]
    h = B.Hist(wl.axes, flags)
    try:
        h.fill(to_device(wl.values), to_device(wl.weights))
        half = n // 2
        h.fill(to_device(np.ascontiguousarray(wl.values[:, :half])), None)  # unit entries add 1 each
        torch.cuda.synchronize()
        got = h.sumw2()
    finally:
        h.close()
    s2, a2 = oracle.sumw2(wl.axes, wl.values, wl.weights)
    c1, _ = oracle.sumw2(wl.axes, np.ascontiguousarray(wl.values[:, :half]), None)
    ref = s2 + c1
    rel = assert_sums_close(got, ref, a2 + c1, RTOL, f"cfg{name} {prec} sumw2")
    print(f"cfg{name} {prec}: max |err| / sum w^2 = {rel:.3g}")


def test_sumw2_requires_flag_and_rejects_batches(B):
    h = B.Hist([W.fixed(10, 0.0, 1.0)])
    h2 = B.Hist([W.fixed(10, 0.0, 1.0)], B.HIST_SUMW2)
    try:
        with pytest.raises(B.HistError) as e:
            h.sumw2()
        assert e.value.code == B.HIST_ERR_STATE
        with pytest.raises(B.HistError) as e:
            B.Batch([h2], [0])
        assert e.value.code == B.HIST_ERR_UNSUPPORTED
        assert not h2.sumw2().any()
    finally:
        h.close()
        h2.close()
