"""Pins of the learned locator's CPU oracle (loss and gradient): a case
worked out by hand and central finite differences of the binary64 loss."""
import numpy as np

from oracle import locator as L


def test_closed_form_one_segment():
    # one segment on [0, 1): u = x, knots K = (1, 3), targets 0 at x = 1/4, 1/2, 3/4:
    # k^ = 1 + 2t -> residuals 1.5, 2, 2.5; L = (2.25 + 4 + 6.25) / 3;
    # dL/dtheta0 = 2/3 * (1.5*0.75 + 2*0.5 + 2.5*0.25) = 2/3 * 2.75,
    # dL/dtheta1 = 2/3 * (1.5*0.25 + 2*0.5 + 2.5*0.75) = 2/3 * 3.25
    loss, g = L.loss_and_grad(1, 0.0, 1.0, [0, 0], [1.0, 3.0], [0.25, 0.5, 0.75], [0.0, 0.0, 0.0])
    assert abs(loss - 12.5 / 3) < 1e-15
    assert abs(g[0] - 2.75 * 2 / 3) < 1e-15 and abs(g[1] - 3.25 * 2 / 3) < 1e-15


def test_segments_and_clamping():
    # below the range -> segment 0 at t = 0; above -> last segment at t = 1
    s, t = L.segments(4, 0.0, 4.0, [-1.0, 0.0, 0.3, 0.99, 5.0])
    assert list(s) == [0, 0, 1, 3, 3]
    assert t[0] == 0.0 and t[-1] == 1.0 and abs(t[2] - 0.2) < 1e-6


def test_trunc24_matches_float32_truncation():
    rng = np.random.default_rng(1)
    x = rng.normal(0, 100, 1000)
    f = L.trunc24(x).astype(np.float64)
    assert np.all(np.abs(f) <= np.abs(x)) and np.all(np.abs(x - f) <= np.abs(x) * 2.0 ** -23)
    assert L.trunc24([0.0])[0] == 0 and L.trunc24([1e300])[0] == np.float32(2.0 ** 127)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    nseg = 16
    x = rng.uniform(-1.0, 3.0, 400)
    y = rng.uniform(0, 50, 400)
    base = np.sort(rng.integers(0, 50, nseg + 1))
    theta = rng.normal(0, 2, nseg + 1)
    u0, us = -1.0, nseg / 4.0
    loss, g = L.loss_and_grad(nseg, u0, us, base, theta, x, y)
    h = 1e-6
    for j in range(nseg + 1):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (L.loss_and_grad(nseg, u0, us, base, tp, x, y)[0] - L.loss_and_grad(nseg, u0, us, base, tm, x, y)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(g[j])), (j, fd, g[j])
