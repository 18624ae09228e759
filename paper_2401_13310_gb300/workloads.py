"""Seeded synthetic workloads shaped like collider event columns.

This module only draws random inputs and builds axis descriptions; it holds
none of the histogramming arithmetic, so both the CUDA path and the CPU
oracle can be fed from it.

Host arrays come from numpy's PCG64 (``numpy.random.default_rng(seed)``);
device arrays, used where the host would take too long to draw them, come from
torch's Philox generator on the GPU with the same seed and the same
distributions (a different stream of numbers).

The workloads echo the benchmark of Sec. 4.2 of the paper (binary64 columns,
1000 bins, millions to a billion events) and widen it with the shapes of
collider data: a Gaussian-core coordinate, an exponentially falling
transverse momentum, a uniform azimuth, a wide pseudorapidity.

Axes are plain dicts: ``{"kind": "fixed", "nbins", "xmin", "xmax"}`` or
``{"kind": "variable", "edges"}``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------- axes -----


def fixed(nbins: int, xmin: float, xmax: float) -> dict:
    return {"kind": "fixed", "nbins": int(nbins), "xmin": float(xmin), "xmax": float(xmax)}


def variable(edges) -> dict:
    e = np.ascontiguousarray(edges, dtype=np.float64)
    if e.ndim != 1 or e.shape[0] < 2 or not np.all(np.diff(e) > 0):
        raise ValueError("edges must be a strictly increasing 1-D array of length >= 2")
    return {"kind": "variable", "edges": e}


def log_edges(nbins: int, lo_exp: float, hi_exp: float) -> np.ndarray:
    """Edges 10**(lo + (hi-lo)*i/nbins), i = 0..nbins (endpoints exact powers)."""
    i = np.arange(nbins + 1, dtype=np.float64)
    return np.power(10.0, lo_exp + (hi_exp - lo_exp) * i / nbins)


def jittered_edges(nbins: int, lo: float, hi: float, rng: np.random.Generator,
                   jitter: float = 0.3) -> np.ndarray:
    """Uniform edges on [lo, hi] with the interior ones moved by up to
    +-jitter of a bin width (so they stay strictly increasing)."""
    w = (hi - lo) / nbins
    k = np.arange(1, nbins, dtype=np.float64)
    inner = lo + (k + rng.uniform(-jitter, jitter, size=nbins - 1)) * w
    return np.concatenate(([lo], inner, [hi]))


# A three-component Gaussian mixture (weights, means, standard deviations).
MIXTURE = ((0.5, 0.3, 0.2), (0.0, 3.0, -4.0), (1.0, 0.5, 2.0))


def mixture_cdf(x: np.ndarray) -> np.ndarray:
    from scipy.special import ndtr
    p, mu, sd = MIXTURE
    return sum(pi * ndtr((x - m) / s) for pi, m, s in zip(p, mu, sd))


def mixture_quantile_edges(nedges: int) -> np.ndarray:
    """Edges at the mixture quantiles (k + 0.5) / nedges, k = 0..nedges-1,
    found by binary64 bisection on the mixture CDF."""
    target = (np.arange(nedges, dtype=np.float64) + 0.5) / nedges
    lo = np.full(nedges, -30.0)
    hi = np.full(nedges, 30.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        below = mixture_cdf(mid) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
        if np.all((hi - lo) <= np.spacing(np.abs(mid)) * 2):
            break
    e = 0.5 * (lo + hi)
    if not np.all(np.diff(e) > 0):
        raise AssertionError("mixture quantile edges are not strictly increasing")
    return e


def mixture_nedges(j: int) -> int:
    return int(round(10 ** (4 + 2 * j / 7)))


# ------------------------------------------------------------ workloads ----


@dataclass
class Workload:
    """One fill: ``values`` has shape (ndim, n) (axis d in row d),
    ``weights`` shape (n,) or None for unit weights."""
    name: str
    axes: list
    values: object
    weights: object = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.values.shape[1])

    @property
    def ndim(self) -> int:
        return len(self.axes)


@dataclass
class BatchWorkload:
    """Many histograms from one event stream: ``columns`` has shape
    (ncols, n); histogram i reads column ``col_of_hist[i]``."""
    name: str
    axes: list            # one 1-D axis per histogram
    col_of_hist: list
    columns: object
    weights: object = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.columns.shape[1])


def _rng(seed):
    return np.random.default_rng(seed)


def _torch_gen(seed, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def cfg1(n: int = 1 << 20, device: str = "cpu", seed: int = 0) -> Workload:
    """1D, 100 fixed bins on [0,1), x ~ U[-0.1, 1.1) (both flow bins hit),
    unit weights."""
    axes = [fixed(100, 0.0, 1.0)]
    if device == "cpu":
        x = _rng(seed).uniform(-0.1, 1.1, size=n)
        vals = x.reshape(1, n)
    else:
        import torch
        g = _torch_gen(seed, device)
        vals = torch.empty((1, n), dtype=torch.float64, device=device).uniform_(-0.1, 1.1, generator=g)
    return Workload("1d_fixed100_unit", axes, vals, None, {"seed": seed})


def cfg2a(n: int = 100_000_000, device: str = "cpu", seed: int = 1) -> Workload:
    """1D weighted: 1000 fixed bins on [-5,5), x ~ N(0,1), w ~ U[0.5,1.5)."""
    axes = [fixed(1000, -5.0, 5.0)]
    if device == "cpu":
        r = _rng(seed)
        vals = r.standard_normal(n).reshape(1, n)
        w = r.uniform(0.5, 1.5, size=n)
    else:
        import torch
        g = _torch_gen(seed, device)
        vals = torch.randn((1, n), dtype=torch.float64, device=device, generator=g)
        w = torch.empty(n, dtype=torch.float64, device=device).uniform_(0.5, 1.5, generator=g)
    return Workload("1d_fixed1000_weighted", axes, vals, w, {"seed": seed})


def cfg2b(n: int = 100_000_000, device: str = "cpu", seed: int = 2) -> Workload:
    """1D weighted: 500 variable bins, edges 10**(3i/500) on [1, 1000],
    x ~ Exponential(mean 30), w ~ U[0.5,1.5)."""
    axes = [variable(log_edges(500, 0.0, 3.0))]
    if device == "cpu":
        r = _rng(seed)
        vals = r.exponential(30.0, size=n).reshape(1, n)
        w = r.uniform(0.5, 1.5, size=n)
    else:
        import torch
        g = _torch_gen(seed, device)
        vals = torch.empty((1, n), dtype=torch.float64, device=device).exponential_(1.0 / 30.0, generator=g)
        w = torch.empty(n, dtype=torch.float64, device=device).uniform_(0.5, 1.5, generator=g)
    return Workload("1d_var500_weighted", axes, vals, w, {"seed": seed})


def cfg3a(n: int = 100_000_000, device: str = "cpu", seed: int = 3) -> Workload:
    """2D 1000 x 1000 fixed bins on [-5,5)^2; (x, y) standard normal with
    correlation 0.6 (y = 0.6 x + 0.8 z); w ~ U[0, 2)."""
    axes = [fixed(1000, -5.0, 5.0), fixed(1000, -5.0, 5.0)]
    if device == "cpu":
        r = _rng(seed)
        x = r.standard_normal(n)
        z = r.standard_normal(n)
        vals = np.empty((2, n))
        vals[0] = x
        vals[1] = 0.6 * x + 0.8 * z
        w = r.uniform(0.0, 2.0, size=n)
    else:
        import torch
        g = _torch_gen(seed, device)
        vals = torch.randn((2, n), dtype=torch.float64, device=device, generator=g)
        vals[1].mul_(0.8).add_(vals[0], alpha=0.6)
        w = torch.empty(n, dtype=torch.float64, device=device).uniform_(0.0, 2.0, generator=g)
    return Workload("2d_fixed1000x1000_weighted", axes, vals, w, {"seed": seed})


def cfg3b(n: int = 100_000_000, device: str = "cpu", seed: int = 4) -> Workload:
    """3D 100 x 100 x 100 fixed bins on [0,1)^3; uniform triples; w ~ U[0,2)."""
    axes = [fixed(100, 0.0, 1.0)] * 3
    if device == "cpu":
        r = _rng(seed)
        vals = r.random((3, n))
        w = r.uniform(0.0, 2.0, size=n)
    else:
        import torch
        g = _torch_gen(seed, device)
        vals = torch.rand((3, n), dtype=torch.float64, device=device, generator=g)
        w = torch.empty(n, dtype=torch.float64, device=device).uniform_(0.0, 2.0, generator=g)
    return Workload("3d_fixed100x100x100_weighted", axes, vals, w, {"seed": seed})


def batch_axes(nhist: int = 64, seed: int = 6):
    """64 histograms with log-spaced bin counts round(10 * 10**(4i/63))
    (10 .. 1e5).  Histogram i reads column i mod 3 (pT, phi, eta); even i
    have fixed bins (pT [0,300), phi [-pi,pi), eta [-5,5)), odd i variable
    ones (pT log-spaced on [1,1000]; phi and eta jittered uniform)."""
    r = _rng(seed)
    axes, cols = [], []
    for i in range(nhist):
        nb = int(round(10 * 10 ** (4 * i / (nhist - 1)))) if nhist > 1 else 10
        c = i % 3
        if i % 2 == 0:
            lo, hi = [(0.0, 300.0), (-math.pi, math.pi), (-5.0, 5.0)][c]
            axes.append(fixed(nb, lo, hi))
        else:
            if c == 0:
                axes.append(variable(log_edges(nb, 0.0, 3.0)))
            elif c == 1:
                axes.append(variable(jittered_edges(nb, -math.pi, math.pi, r)))
            else:
                axes.append(variable(jittered_edges(nb, -5.0, 5.0, r)))
        cols.append(c)
    return axes, cols


def cfg4(n: int = 50_000_000, device: str = "cpu", seed: int = 5, nhist: int = 64) -> BatchWorkload:
    """Batched: columns pT ~ Exp(mean 30), phi ~ U[-pi, pi), eta ~ N(0, 2.5);
    w ~ U[0.5, 1.5); 64 histograms (see batch_axes)."""
    axes, cols = batch_axes(nhist)
    if device == "cpu":
        r = _rng(seed)
        c = np.empty((3, n))
        c[0] = r.exponential(30.0, size=n)
        c[1] = r.uniform(-math.pi, math.pi, size=n)
        c[2] = 2.5 * r.standard_normal(n)
        w = r.uniform(0.5, 1.5, size=n)
    else:
        import torch
        g = _torch_gen(seed, device)
        c = torch.empty((3, n), dtype=torch.float64, device=device)
        c[0].exponential_(1.0 / 30.0, generator=g)
        c[1].uniform_(-math.pi, math.pi, generator=g)
        c[2].normal_(0.0, 2.5, generator=g)
        w = torch.empty(n, dtype=torch.float64, device=device).uniform_(0.5, 1.5, generator=g)
    return BatchWorkload("batched64_pt_phi_eta", axes, cols, c, w, {"seed": seed})


def learned_axes(nhist: int = 8, scale: float = 1.0):
    """8 variable axes with round(10**(4 + 2j/7)) edges (1e4 .. 1e6) at the
    quantiles of the Gaussian mixture; ``scale`` < 1 shrinks the edge counts
    for quick tests."""
    return [variable(mixture_quantile_edges(max(16, int(round(mixture_nedges(j) * scale)))))
            for j in range(nhist)]


def mixture_values(n: int, device: str = "cpu", seed: int = 7):
    p, mu, sd = MIXTURE
    if device == "cpu":
        r = _rng(seed)
        u = r.random(n)
        z = r.standard_normal(n)
        comp = (u >= p[0]).astype(np.int64) + (u >= p[0] + p[1]).astype(np.int64)
        m = np.asarray(mu)[comp]
        s = np.asarray(sd)[comp]
        return (m + s * z).reshape(1, n)
    import torch
    g = _torch_gen(seed, device)
    u = torch.rand(n, dtype=torch.float64, device=device, generator=g)
    out = torch.randn((1, n), dtype=torch.float64, device=device, generator=g)
    comp = (u >= p[0]).to(torch.int64) + (u >= p[0] + p[1]).to(torch.int64)
    del u
    m = torch.tensor(mu, dtype=torch.float64, device=device)[comp]
    s = torch.tensor(sd, dtype=torch.float64, device=device)[comp]
    del comp
    out[0].mul_(s).add_(m)
    return out


def cfg5(n: int = 1_000_000_000, device: str = "cpu", seed: int = 7, nhist: int = 8,
         scale: float = 1.0) -> BatchWorkload:
    """Learned locator: one column of mixture draws filled (unit weights)
    into 8 variable-edge histograms with edges at the mixture quantiles."""
    axes = learned_axes(nhist, scale)
    vals = mixture_values(n, device, seed)
    return BatchWorkload("learned8_mixture_quantiles", axes, [0] * nhist, vals, None,
                         {"seed": seed})


CONFIGS = {"1": cfg1, "2a": cfg2a, "2b": cfg2b, "3a": cfg3a, "3b": cfg3b, "4": cfg4, "5": cfg5}
