"""Per-bin sum of squared weights (HIST_SUMW2, ROOT's Sumw2) against the
oracle, in every precision mode, for shared-memory bins (compensated FP32
words) and global bins (binary64 atomics), unit and weighted fills mixed.
Bound per bin, A = sum w^2 of its entries, m <= its entry count, B <= 1216
blocks:  |err| <= 2^-44 A + 2^-48 ((m + 1)^2 + 1) A + B 2^-53 A."""
import numpy as np
import pytest

import oracle
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


def _bound(counts, A):
    m = counts.astype(np.float64)
    return 2.0 ** -44 * A + 2.0 ** -48 * ((m + 1.0) ** 2 + 1.0) * A + 1216 * 2.0 ** -53 * A


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
    counts = oracle.fill(wl.axes, wl.values, wl.weights).counts
    err = np.abs(got - ref)
    bound = _bound(counts, a2) + 1e-300
    assert np.all(err <= bound), f"cfg{name} {prec}: worst error/bound {np.max(err / bound):.3g}"
    print(f"cfg{name} {prec}: max |err| / sum w^2 = {np.max(err / np.maximum(a2 + c1, 1e-300)):.3g}")


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
