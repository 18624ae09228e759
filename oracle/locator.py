"""CPU oracle of the learned bin locator's training loss and gradient.

TEST INFRASTRUCTURE.  Only the tests import this module.  It restates, in
plain numpy binary64, the model and loss that the library documents for its
learned locator (the paper has no such component; the locator is an index
model in the spirit of learned index structures, corrected by an exact
search):

  xf  = the coordinate truncated to 24 significant bits (an FP32 value;
        +-0 below 2^-126, +-2^127 at or above 2^128)
  u   = fl32(fl32(xf - u0) * u_scale), clamped below at 0
  s   = min(floor(u), nseg - 1),   t = min(u - s, 1)       (segment, position)
  K_j = base_j + theta_j                                      (knot values)
  k^  = K_s (1 - t) + K_{s+1} t                               (real arithmetic here)
  L   = (1/N) sum_i (k^_i - y_i)^2
  dL/dtheta_j = (2/N) sum_i r_i [ (1 - t_i) [s_i = j] + t_i [s_i + 1 = j] ]

u and t are computed in FP32 exactly as defined, so both sides assign the
same segment to each sample; k^, the residuals, the loss and the gradient
are binary64 here.
"""
from __future__ import annotations

import numpy as np


def trunc24(x) -> np.ndarray:
    """binary64 -> FP32 by truncating the significand to 24 bits (saturating)."""
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    e = (hi >> np.uint32(20)) & np.uint32(0x7FF)
    f = ((b >> np.uint64(29)).astype(np.uint32) - np.uint32(0xC0000000)) & np.uint32(0x7FFFFFFF)
    f = np.where(e < 897, np.uint32(0), f)
    f = np.where(e > 1150, np.uint32(0x7F000000), f)
    f = f | (hi & np.uint32(0x80000000))
    return f.astype(np.uint32).view(np.float32)


def segments(nseg: int, u0: float, u_scale: float, x):
    """Segment index s and in-segment position t of every coordinate."""
    xf = trunc24(x)
    u = (xf - np.float32(u0)).astype(np.float32) * np.float32(u_scale)
    u = np.maximum(u.astype(np.float32), np.float32(0.0))
    s = np.minimum(np.floor(u), np.float32(nseg - 1)).astype(np.int64)
    t = np.minimum((u - s.astype(np.float32)).astype(np.float32), np.float32(1.0))
    return s, t.astype(np.float64)


def loss_and_grad(nseg: int, u0: float, u_scale: float, base, theta, x, target):
    """Mean squared index error and its gradient with respect to theta."""
    base = np.asarray(base, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    y = np.asarray(target, dtype=np.float64)
    s, t = segments(nseg, u0, u_scale, x)
    K = base + theta
    khat = K[s] * (1.0 - t) + K[s + 1] * t
    r = khat - y
    n = r.shape[0]
    loss = float(np.sum(r * r) / n)
    grad = np.zeros(nseg + 1)
    np.add.at(grad, s, 2.0 * r * (1.0 - t) / n)
    np.add.at(grad, s + 1, 2.0 * r * t / n)
    return loss, grad
