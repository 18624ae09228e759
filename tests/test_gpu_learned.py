"""The learned locator on the GPU: its training gradients against the CPU
oracle, its certified window, bit-exact bins with the model installed, and
what training gains over the untrained (interpolating) model."""
import math

import numpy as np
import pytest

import oracle
from oracle import locator as OL
from paper_2401_13310_gb300 import workloads as W
from tests.helpers import edge_probe_values, gpu_fill, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2401_13310_gb300 import _build
    _build.build()
    from paper_2401_13310_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("nseg", [1, 16, 256])
def test_gradients_match_cpu_oracle(B, nseg):
    rng = np.random.default_rng(nseg)
    n = 20_000
    x = rng.uniform(-2.0, 6.0, n)
    y = rng.uniform(0, 400, n).astype(np.float32)
    base = np.sort(rng.integers(0, 400, nseg + 1)).astype(np.int32)
    theta = rng.normal(0, 3, nseg + 1).astype(np.float32)
    u0 = np.float32(-2.0)
    us = np.float32(nseg / 8.0)
    loss_g, grad_g = B.hist_locator_loss_grad(nseg, float(u0), float(us), base, theta, x, y)
    loss_c, grad_c = OL.loss_and_grad(nseg, float(u0), float(us), base, theta.astype(np.float64), x, y)
    assert abs(loss_g - loss_c) <= 1e-5 * loss_c
    scale = np.max(np.abs(grad_c))
    assert np.max(np.abs(grad_g - grad_c)) <= 1e-4 * scale, np.max(np.abs(grad_g - grad_c)) / scale


def _mixture_axis(nedges):
    return W.variable(W.mixture_quantile_edges(nedges))


@pytest.mark.parametrize("nedges", [1000, 20_000])
def test_learned_locate_bit_exact(B, nedges):
    import torch
    axis = _mixture_axis(nedges)
    h = B.Hist([axis])
    try:
        rep = h.train_locator(0)
        assert rep["loss"] < rep["loss_untrained"]  # training lowers the objective
        assert 0 <= rep["window"] <= 8
        rng = np.random.default_rng(3)
        T = B.hist_axis_thresholds(axis)
        x = np.concatenate([edge_probe_values(axis, T, rng, nrand=5000),
                            W.mixture_values(200_000, seed=9)[0]])
        got = h.locate(to_device(x.reshape(1, -1))).cpu().numpy()
        torch.cuda.synchronize()
    finally:
        h.close()
    ref = oracle.locate([axis], x.reshape(1, -1))
    assert np.array_equal(got, ref), f"{np.count_nonzero(got != ref)} mismatches"
    print(f"nedges={nedges}: {rep}")


def _time_fill(B, axis, x, learned, reps=5, flags=None):
    import torch
    h = B.Hist([axis], B.HIST_LOCATOR_BSEARCH if flags is None else flags)
    try:
        if learned:
            h.train_locator(0)
        for _ in range(2):
            h.fill(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            h.fill(x)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, h.counts()
    finally:
        h.close()


@pytest.mark.parametrize("nedges", [100_000, 1_000_000])
def test_learned_locator_gain_over_binary_search(B, nedges):
    """What the trained model gains over the method without it: the same
    exact counts, filled faster than by binary search over the edges."""
    axis = _mixture_axis(nedges)
    x = W.mixture_values(20_000_000, device="cuda", seed=13)
    t_bs, c_bs = _time_fill(B, axis, x, learned=False)
    t_lm, c_lm = _time_fill(B, axis, x, learned=True)
    t_bk, c_bk = _time_fill(B, axis, x, learned=False, flags=B.HIST_LOCATOR_AUTO)
    assert np.array_equal(c_bs, c_lm)
    assert np.array_equal(c_bs, c_bk)
    print(f"nedges={nedges}: binary search {t_bs:.3f} ms, learned {t_lm:.3f} ms, gain {t_bs / t_lm:.2f}x; "
          f"default locator {t_bk:.3f} ms")
    assert t_lm < t_bs


def test_learned_fill_matches_oracle(B):
    import torch
    axis = _mixture_axis(5000)
    x = W.mixture_values(300_001, seed=11)
    w = np.random.default_rng(5).uniform(0.5, 1.5, 300_001)
    for weights in (None, w):
        h = B.Hist([axis], B.HIST_TRACK_COUNTS)
        try:
            h.train_locator(0)
            h.fill(to_device(x), to_device(weights))
            bins, stats = h.result()
            counts = h.counts()
        finally:
            h.close()
        ref = oracle.fill([axis], x, weights)
        assert np.array_equal(counts, ref.counts)
        if weights is None:
            assert np.array_equal(bins, ref.counts.astype(np.float64))
        else:
            assert np.all(np.abs(bins - ref.bins_acc) <= 1e-12 * ref.bins_abs)
        assert np.all(np.abs(stats[1:] - ref.stats_acc[1:]) <= 1e-12 * ref.stats_abs[1:])


def test_train_locator_rejects_fixed_axis(B):
    h = B.Hist([W.fixed(10, 0.0, 1.0)])
    try:
        with pytest.raises(B.HistError) as e:
            h.train_locator(0)
        assert e.value.code == B.HIST_ERR_ARG
    finally:
        h.close()
