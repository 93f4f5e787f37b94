"""Seeded synthetic inputs for the signature-kernel PDE solve.

This module is shared by the CUDA path's tests and benchmark and by the FP64
CPU oracle.  It holds none of the method's arithmetic: it only draws paths.

Every workload is drawn in float64 with numpy's PCG64 from a fixed seed and
``SeedSequence.spawn`` sub-seeds, one per tensor.  The FP32 runs use the cast
``.astype(float32)``; the oracle is then run on that cast promoted back to
float64, so a parity error measures the algorithm, not input rounding.

Shapes follow the paper's workloads (Sec. 3.1.1: piecewise-linear
interpolations of Brownian paths, rescaled to O(1) amplitude as Sec. 3.1
advises).  A path has L points in d channels; ``d`` counts every channel,
including the time channel where there is one.
"""
from __future__ import annotations

import numpy as np

SEEDS = {1: 2006_0001, 2: 2006_0002, 3: 2006_0003, 4: 2006_0004, 5: 2006_0005}


def _rngs(seed: int, n: int):
    return [np.random.Generator(np.random.PCG64(s))
            for s in np.random.SeedSequence(seed).spawn(n)]


def brownian(rng, B: int, L: int, d: int, step_var: float, time_channel: bool):
    """B paths of L points: optional time channel t_i = i/(L-1), then walks
    w_0 = 0, w_i = sum_{k<i} xi_k with xi ~ N(0, step_var)."""
    nw = d - 1 if time_channel else d
    xi = rng.normal(0.0, np.sqrt(step_var), size=(B, max(L - 1, 0), nw))
    w = np.zeros((B, L, nw))
    if L > 1:
        w[:, 1:, :] = np.cumsum(xi, axis=1)
    if not time_channel:
        return w
    t = np.broadcast_to((np.arange(L) / max(L - 1, 1))[None, :, None], (B, L, 1))
    return np.concatenate([t, w], axis=2)


def straight_lines(rng, B: int, L: int, d: int, scale: float = 1.0 / 3.0):
    """Pairs of straight lines x_i = a t_i, y_i = b t_i, t_i = i/(L-1),
    with a, b ~ N(0, scale * I_d)."""
    a = rng.normal(0.0, np.sqrt(scale), size=(B, d))
    b = rng.normal(0.0, np.sqrt(scale), size=(B, d))
    t = np.arange(L) / max(L - 1, 1)
    return (a[:, None, :] * t[None, :, None], b[:, None, :] * t[None, :, None], a, b)


def gram_small(seed: int = SEEDS[1]):
    """Gram 8x8, L=M=32, d=3 (time + 2 walks, xi ~ N(0, 1/L)), dyadic order 1,
    plus 8 straight-line pairs (a, b ~ N(0, I/3)) for the closed-form check."""
    r = _rngs(seed, 3)
    X = brownian(r[0], 8, 32, 3, 1.0 / 32, True)
    Y = brownian(r[1], 8, 32, 3, 1.0 / 32, True)
    xs, ys, a, b = straight_lines(r[2], 8, 32, 3)
    return dict(X=X, Y=Y, lines_x=xs, lines_y=ys, a=a, b=b, dyadic_order=1)


def gram_256(seed: int = SEEDS[2], B: int = 256, L: int = 128):
    """Gram 256x256, L=M=128, d=8 (time + 7 walks, xi ~ N(0, 1/(L d))),
    dyadic order 2."""
    d = 8
    r = _rngs(seed, 2)
    X = brownian(r[0], B, L, d, 1.0 / (L * d), True)
    Y = brownian(r[1], B, L, d, 1.0 / (L * d), True)
    return dict(X=X, Y=Y, dyadic_order=2)


def uneven_pairs(seed: int = SEEDS[3], B: int = 4096, lo: int = 16, hi: int = 512, d: int = 16):
    """B independent pairs with lengths L, M ~ Uniform{lo..hi}, d walks with
    xi ~ N(0, 1/(L d)) (no time channel), dyadic order 1.  Returned packed:
    Xp [sum L, d] with offsets x_off [B+1], likewise for Y."""
    r = _rngs(seed, 3)
    Ls = r[0].integers(lo, hi + 1, size=B)
    Ms = r[0].integers(lo, hi + 1, size=B)
    xs = [brownian(r[1], 1, int(L), d, 1.0 / (int(L) * d), False)[0] for L in Ls]
    ys = [brownian(r[2], 1, int(M), d, 1.0 / (int(M) * d), False)[0] for M in Ms]
    x_off = np.zeros(B + 1, np.int64)
    y_off = np.zeros(B + 1, np.int64)
    x_off[1:] = np.cumsum(Ls)
    y_off[1:] = np.cumsum(Ms)
    return dict(Xp=np.concatenate(xs, 0), Yp=np.concatenate(ys, 0),
                x_off=x_off, y_off=y_off, dyadic_order=1)


def mmd_batches(seed: int = SEEDS[4], B: int = 128, L: int = 256, d: int = 32, drift: float = 0.1):
    """Two batches of B paths, L points, d walks with xi ~ N(0, 1/(L d));
    Y gets a drift of `drift` per unit time in every channel (y_i += drift t_i),
    dyadic order 1."""
    r = _rngs(seed, 2)
    X = brownian(r[0], B, L, d, 1.0 / (L * d), False)
    Y = brownian(r[1], B, L, d, 1.0 / (L * d), False)
    t = np.arange(L) / (L - 1)
    Y = Y + drift * t[None, :, None]
    return dict(X=X, Y=Y, dyadic_order=1)


def long_pairs(seed: int = SEEDS[5], B: int = 64, L: int = 4096, d: int = 64):
    """B pairs, L=M=4096, d=64 (time + 63 walks, xi ~ N(0, 1/(L d))),
    dyadic order 0 and 1."""
    r = _rngs(seed, 2)
    X = brownian(r[0], B, L, d, 1.0 / (L * d), True)
    Y = brownian(r[1], B, L, d, 1.0 / (L * d), True)
    return dict(X=X, Y=Y, dyadic_orders=(0, 1))


def fbm_paths(seed: int = 2006_0006, B: int = 30, L: int = 64, hursts=(0.2, 0.5, 0.8)):
    """The support-reduction example of Sec. 5.3: B sample paths of fractional
    Brownian motion on [0, 1], each with a Hurst exponent drawn uniformly from
    `hursts`, time-augmented (d = 2: t, B^H_t), L points.  Drawn exactly on
    the grid t_i = i / (L - 1) from the covariance
    1/2 (s^2H + t^2H - |s - t|^2H) by its Cholesky factor.  Returns (paths
    [B, L, 2], the Hurst exponent of each path)."""
    r = _rngs(seed, 2)
    H = r[0].choice(np.asarray(hursts, dtype=np.float64), size=B)
    t = np.linspace(0.0, 1.0, L)
    s, u = np.meshgrid(t[1:], t[1:], indexing="ij")
    X = np.zeros((B, L, 2))
    X[:, :, 0] = t
    for b in range(B):
        h2 = 2.0 * H[b]
        C = 0.5 * (s ** h2 + u ** h2 - np.abs(s - u) ** h2)
        Lc = np.linalg.cholesky(C + 1e-12 * np.eye(L - 1))
        X[b, 1:, 1] = Lc @ r[1].standard_normal(L - 1)
    return X, H


def random_paths(seed: int, B: int, L: int, d: int, scale: float = 1.0, time_channel: bool = False):
    """Generic seeded paths for tests: walks with xi ~ N(0, scale^2/(L d))."""
    r = _rngs(seed, 1)[0]
    return brownian(r, B, L, d, scale * scale / (max(L, 1) * d), time_channel)


def f32(a):
    """The FP32 cast given to the GPU, and its exact FP64 promotion for the
    oracle."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    return a32, a32.astype(np.float64)
