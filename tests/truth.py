"""Independent ground truth for pinning the oracle (test helpers only).

Nothing here runs the finite-difference scheme.  It computes the TRUE
signature kernel <S(x), S(y)> of piecewise-linear paths by other routes:

* ``sig_truncated``: the truncated signature of a piecewise-linear path as
  the tensor product of the segment exponentials exp(dx_1) (x) ... (x) exp(dx_n)
  (Chen's identity, Appendix B; a linear segment's signature is the tensor
  exponential of its increment, Thm. "universal"), truncated at level N.
* ``sig_inner``: <S(x), S(y)> = sum over levels of the Euclidean inner product
  of the level-k tensors (the inner product on T(V), Sec. 2.1), with the
  factorial-decay bound on the neglected levels (Sec. 2.1).
* ``series_I0``: sum_k c^k / (k!)^2 = I_0(2 sqrt c) (c >= 0) or J_0(2 sqrt|c|)
  (c < 0), the Riemann function of the constant-coefficient Goursat problem
  (Appendix A), evaluated by its power series.
"""
from __future__ import annotations

import math

import numpy as np


def series_I0(c: float, terms: int = 80) -> float:
    s, t = 1.0, 1.0
    for k in range(1, terms):
        t *= c / (k * k)
        s += t
    return s


def _tensor_mul(a, b, N, d):
    out = [np.zeros(d ** n) for n in range(N + 1)]
    for i in range(N + 1):
        for j in range(N + 1 - i):
            out[i + j] += np.outer(a[i], b[j]).ravel()
    return out


def _seg_exp(dx, N):
    lv = [np.ones(1)]
    for n in range(1, N + 1):
        lv.append(np.outer(lv[-1], dx).ravel() / n)
    return lv


def sig_truncated(x, N: int):
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    S = [np.ones(1)] + [np.zeros(d ** n) for n in range(1, N + 1)]
    for p in range(x.shape[0] - 1):
        S = _tensor_mul(S, _seg_exp(x[p + 1] - x[p], N), N, d)
    return S


def sig_inner(x, y, N: int):
    """Returns (sum_{k<=N} <S^k(x), S^k(y)>, bound on the neglected tail)."""
    Sx, Sy = sig_truncated(x, N), sig_truncated(y, N)
    val = sum(float(a @ b) for a, b in zip(Sx, Sy))
    lx = float(np.abs(np.diff(x, axis=0)).sum())   # 1-variation in the l1 norm >= the l2 one
    ly = float(np.abs(np.diff(y, axis=0)).sum())
    tail = sum((lx * ly) ** k / math.factorial(k) ** 2 for k in range(N + 1, N + 40))
    return val, tail


def richardson(k_lam, k_lam1):
    """Eliminates the 4^-lambda leading error term (global error theorem, Sec. 3.1)."""
    return (4.0 * k_lam1 - k_lam) / 3.0
