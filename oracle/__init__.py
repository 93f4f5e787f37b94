"""FP64 CPU oracle of the signature-kernel PDE solve — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never imports it
and shares no code with it (only the seeded input generators are common).

The arithmetic lives in ``sigk_oracle.c`` (plain C, float64, no FMA
contraction), which follows Sec. 3.1 of the paper: the explicit
finite-difference scheme on the dyadically refined grid P_lambda with the
refined increment inner product 2^(-2 lambda) <dx_p, dy_q>, boundary value 1,
and the kernel read at the terminal corner.  ``mmd2`` is the unbiased MMD
estimator named in Sec. 3.1.1, written as the usual U-statistic.

Pins (tests/test_oracle_pins.py) tie it to closed forms, brute-force truncated
signatures, invariants and finite differences.  Every function is pinned.

Every entry point also takes ``scheme`` ("explicit", or "implicit": the
four-point quadrature of the remark after the scheme in Sec. 3.1) and
``static_kernel`` ("linear", or "rbf" with bandwidth ``sigma``: the PDE of the
paths lifted by a static kernel, Sec. 2.2).

``support_reduction`` is the proximal gradient iteration of Sec. 5.3 on a
given Gram matrix (numpy float64, one matrix-vector product per step).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_sigk_pair.restype = ctypes.c_double
        L.oracle_sigk_pair.argtypes = [_dp, _i64, _dp, _i64, _i64, ctypes.c_int]
        L.oracle_sigk_pairs.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, ctypes.c_int, _dp]
        L.oracle_sigk_gram.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _i64, ctypes.c_int, _dp]
        L.oracle_sigk_pairs_varlen.argtypes = [_dp, _ip, _dp, _ip, _i64, _i64, ctypes.c_int, _dp]
        L.oracle_sigk_pair_grad.restype = ctypes.c_double
        L.oracle_sigk_pair_grad.argtypes = [_dp, _i64, _dp, _i64, _i64, ctypes.c_int,
                                            ctypes.c_double, _dp, _dp]
        L.oracle_sigk_pairs_grad.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, ctypes.c_int,
                                             _dp, _dp, _dp]
        L.oracle_sigk_gram_grad.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _i64, ctypes.c_int,
                                            _dp, _dp, _dp]
        _dbl, _int = ctypes.c_double, ctypes.c_int
        L.oracle_sigk_pair_ex.restype = _dbl
        L.oracle_sigk_pair_ex.argtypes = [_dp, _i64, _dp, _i64, _i64, _int, _int, _int, _dbl]
        L.oracle_sigk_pairs_ex.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _int, _int, _int, _dbl, _dp]
        L.oracle_sigk_gram_ex.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _i64, _int, _int, _int,
                                          _dbl, _dp]
        L.oracle_sigk_pairs_varlen_ex.argtypes = [_dp, _ip, _dp, _ip, _i64, _i64, _int, _int, _int,
                                                  _dbl, _dp]
        L.oracle_sigk_pair_grad_ex.restype = _dbl
        L.oracle_sigk_pair_grad_ex.argtypes = [_dp, _i64, _dp, _i64, _i64, _int, _int, _int, _dbl,
                                               _dbl, _dp, _dp]
        L.oracle_sigk_pairs_grad_ex.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _int, _int, _int,
                                                _dbl, _dp, _dp, _dp]
        L.oracle_sigk_gram_grad_ex.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _i64, _int, _int,
                                               _int, _dbl, _dp, _dp, _dp]
        L.oracle_sigk_pair_surface.restype = _dbl
        L.oracle_sigk_pair_surface.argtypes = [_dp, _i64, _dp, _i64, _i64, _int, _int, _int, _dbl, _dp]
        L.oracle_sigk_pairs_surface.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _int, _int, _int,
                                                _dbl, _dp, _dp]
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


SCHEMES = {"explicit": 0, "implicit": 1}
STATIC_KERNELS = {"linear": 0, "rbf": 1}


def _variant(scheme, static_kernel, sigma):
    """(scheme code, kernel code, sigma); None for the paper's main variant
    (explicit scheme, linear kernel), which runs the original entry points."""
    sc, kc = SCHEMES[scheme], STATIC_KERNELS[static_kernel]
    if kc == 1 and not sigma > 0:
        raise ValueError("the RBF kernel needs sigma > 0")
    if sc == 0 and kc == 0:
        return None
    return sc, kc, float(sigma)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def sigkernel(x, y, dyadic_order: int, scheme="explicit", static_kernel="linear",
              sigma=1.0) -> float:
    """k_{x,y} on P_lambda for one pair; x: [L,d], y: [M,d]."""
    x, xp = _d(x)
    y, yp = _d(y)
    assert x.ndim == 2 and y.ndim == 2 and x.shape[1] == y.shape[1]
    v = _variant(scheme, static_kernel, sigma)
    if v is not None:
        return float(lib().oracle_sigk_pair_ex(xp, x.shape[0], yp, y.shape[0], x.shape[1],
                                               int(dyadic_order), *v))
    return float(lib().oracle_sigk_pair(xp, x.shape[0], yp, y.shape[0], x.shape[1],
                                        int(dyadic_order)))


def surface(x, y, dyadic_order: int, scheme="explicit", static_kernel="linear", sigma=1.0):
    """The scheme's solution at the sample-grid nodes (P_0 inside P_lambda):
    [L, M] with surf[i, j] ~ k_{x,y}(s_i, t_j); row and column 0 are 1."""
    x, xp = _d(x)
    y, yp = _d(y)
    sc, kc = SCHEMES[scheme], STATIC_KERNELS[static_kernel]
    if kc == 1 and not sigma > 0:
        raise ValueError("the RBF kernel needs sigma > 0")
    out = np.empty((x.shape[0], y.shape[0]))
    lib().oracle_sigk_pair_surface(xp, x.shape[0], yp, y.shape[0], x.shape[1], int(dyadic_order), sc,
                                   kc, float(sigma), out.ctypes.data_as(_dp))
    return out


def pairs_surface(X, Y, dyadic_order: int, scheme="explicit", static_kernel="linear", sigma=1.0):
    """(k [B], surfaces [B, L, M]) for pairs (X_b, Y_b)."""
    X, xp = _d(X)
    Y, yp = _d(Y)
    B, L, d = X.shape
    M = Y.shape[1]
    sc, kc = SCHEMES[scheme], STATIC_KERNELS[static_kernel]
    if kc == 1 and not sigma > 0:
        raise ValueError("the RBF kernel needs sigma > 0")
    out = np.empty(B)
    surf = np.empty((B, L, M))
    lib().oracle_sigk_pairs_surface(xp, yp, B, L, M, d, int(dyadic_order), sc, kc, float(sigma),
                                    out.ctypes.data_as(_dp), surf.ctypes.data_as(_dp))
    return out, surf


def pairs(X, Y, dyadic_order: int, scheme="explicit", static_kernel="linear", sigma=1.0):
    """out[b] = k(X_b, Y_b); X: [B,L,d], Y: [B,M,d]."""
    X, xp = _d(X)
    Y, yp = _d(Y)
    B, L, d = X.shape
    out = np.empty(B)
    v = _variant(scheme, static_kernel, sigma)
    if v is not None:
        lib().oracle_sigk_pairs_ex(xp, yp, B, L, Y.shape[1], d, int(dyadic_order), *v,
                                   out.ctypes.data_as(_dp))
        return out
    lib().oracle_sigk_pairs(xp, yp, B, L, Y.shape[1], d, int(dyadic_order),
                            out.ctypes.data_as(_dp))
    return out


def gram(X, Y, dyadic_order: int, scheme="explicit", static_kernel="linear", sigma=1.0):
    """out[i,j] = k(X_i, Y_j)."""
    X, xp = _d(X)
    Y, yp = _d(Y)
    Bx, L, d = X.shape
    By, M, _ = Y.shape
    out = np.empty((Bx, By))
    v = _variant(scheme, static_kernel, sigma)
    if v is not None:
        lib().oracle_sigk_gram_ex(xp, yp, Bx, By, L, M, d, int(dyadic_order), *v,
                                  out.ctypes.data_as(_dp))
        return out
    lib().oracle_sigk_gram(xp, yp, Bx, By, L, M, d, int(dyadic_order), out.ctypes.data_as(_dp))
    return out


def pairs_varlen(Xp, x_off, Yp, y_off, dyadic_order: int, scheme="explicit",
                 static_kernel="linear", sigma=1.0):
    """Pairs of uneven lengths, packed as [sum L, d] with offsets [B+1]."""
    Xp, xp = _d(Xp)
    Yp, yp = _d(Yp)
    xo = np.ascontiguousarray(x_off, dtype=np.int64)
    yo = np.ascontiguousarray(y_off, dtype=np.int64)
    B = xo.shape[0] - 1
    out = np.empty(B)
    v = _variant(scheme, static_kernel, sigma)
    if v is not None:
        lib().oracle_sigk_pairs_varlen_ex(xp, xo.ctypes.data_as(_ip), yp, yo.ctypes.data_as(_ip),
                                          B, Xp.shape[1], int(dyadic_order), *v,
                                          out.ctypes.data_as(_dp))
        return out
    lib().oracle_sigk_pairs_varlen(xp, xo.ctypes.data_as(_ip), yp, yo.ctypes.data_as(_ip), B,
                                   Xp.shape[1], int(dyadic_order), out.ctypes.data_as(_dp))
    return out


def sigkernel_grad(x, y, dyadic_order: int, gout: float = 1.0, scheme="explicit",
                   static_kernel="linear", sigma=1.0):
    """(k, dk/dx, dk/dy) for one pair (reverse-mode of the discrete scheme)."""
    x, xp = _d(x)
    y, yp = _d(y)
    dx = np.zeros_like(x)
    dy = np.zeros_like(y)
    v = _variant(scheme, static_kernel, sigma)
    if v is not None:
        k = lib().oracle_sigk_pair_grad_ex(xp, x.shape[0], yp, y.shape[0], x.shape[1],
                                           int(dyadic_order), *v, float(gout),
                                           dx.ctypes.data_as(_dp), dy.ctypes.data_as(_dp))
        return float(k), dx, dy
    k = lib().oracle_sigk_pair_grad(xp, x.shape[0], yp, y.shape[0], x.shape[1],
                                    int(dyadic_order), float(gout), dx.ctypes.data_as(_dp),
                                    dy.ctypes.data_as(_dp))
    return float(k), dx, dy


def pairs_grad(X, Y, dyadic_order: int, gout, scheme="explicit", static_kernel="linear",
               sigma=1.0):
    X, xp = _d(X)
    Y, yp = _d(Y)
    g, gp = _d(gout)
    dX = np.zeros_like(X)
    dY = np.zeros_like(Y)
    B, L, d = X.shape
    v = _variant(scheme, static_kernel, sigma)
    if v is not None:
        lib().oracle_sigk_pairs_grad_ex(xp, yp, B, L, Y.shape[1], d, int(dyadic_order), *v, gp,
                                        dX.ctypes.data_as(_dp), dY.ctypes.data_as(_dp))
        return dX, dY
    lib().oracle_sigk_pairs_grad(xp, yp, B, L, Y.shape[1], d, int(dyadic_order), gp,
                                 dX.ctypes.data_as(_dp), dY.ctypes.data_as(_dp))
    return dX, dY


def gram_grad(X, Y, dyadic_order: int, gout, want_dx: bool = True, want_dy: bool = True,
              scheme="explicit", static_kernel="linear", sigma=1.0):
    X, xp = _d(X)
    Y, yp = _d(Y)
    g, gp = _d(gout)
    Bx, L, d = X.shape
    By, M, _ = Y.shape
    dX = np.zeros_like(X) if want_dx else None
    dY = np.zeros_like(Y) if want_dy else None
    v = _variant(scheme, static_kernel, sigma)
    if v is not None:
        lib().oracle_sigk_gram_grad_ex(xp, yp, Bx, By, L, M, d, int(dyadic_order), *v, gp,
                                       dX.ctypes.data_as(_dp) if want_dx else None,
                                       dY.ctypes.data_as(_dp) if want_dy else None)
        return dX, dY
    lib().oracle_sigk_gram_grad(xp, yp, Bx, By, L, M, d, int(dyadic_order), gp,
                                dX.ctypes.data_as(_dp) if want_dx else None,
                                dY.ctypes.data_as(_dp) if want_dy else None)
    return dX, dY


def mmd2(X, Y, dyadic_order: int) -> float:
    """Unbiased MMD^2 estimator (Sec. 3.1.1 names it; U-statistic form):
    1/(m(m-1)) sum_{i!=j} k(x_i,x_j) + 1/(n(n-1)) sum_{i!=j} k(y_i,y_j)
    - 2/(mn) sum_{i,j} k(x_i,y_j)."""
    m, n = X.shape[0], Y.shape[0]
    Kxx = gram(X, X, dyadic_order)
    Kyy = gram(Y, Y, dyadic_order)
    Kxy = gram(X, Y, dyadic_order)
    sxx = Kxx.sum() - np.trace(Kxx)
    syy = Kyy.sum() - np.trace(Kyy)
    return float(sxx / (m * (m - 1)) + syy / (n * (n - 1)) - 2.0 * Kxy.sum() / (m * n))


def mmd2_grad_x(X, Y, dyadic_order: int):
    """d MMD^2 / dX for the estimator above (X appears in Kxx twice and in Kxy)."""
    m, n = X.shape[0], Y.shape[0]
    gxx = np.full((m, m), 1.0 / (m * (m - 1)))
    np.fill_diagonal(gxx, 0.0)
    dXa, dXb = gram_grad(X, X, dyadic_order, gxx)
    gxy = np.full((m, n), -2.0 / (m * n))
    dXc, _ = gram_grad(X, Y, dyadic_order, gxy, want_dy=False)
    return dXa + dXb + dXc


def soft_threshold(v, tau):
    """The soft-thresholding operator of Sec. 5.3, A_tau(v)_i = v_i - tau if
    v_i > tau, 0 if |v_i| <= tau, v_i + tau if v_i < -tau."""
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    out[v > tau] = v[v > tau] - tau
    out[v < -tau] = v[v < -tau] + tau
    return out


def support_reduction(K, alpha, beta0, gamma: float, lam: float, iters: int):
    """Proximal gradient descent for min_beta L(beta) + lam |beta|_1 with
    L(beta) = sum_ij (alpha_i - beta_i)(alpha_j - beta_j) K_ij (Sec. 5.3):
      beta <- A_{gamma lam}(beta - gamma grad L(beta)),  grad L = -2 K (alpha - beta)
    (the soft threshold at gamma lam is the proximal map of gamma lam |.|_1).
    Returns (beta after `iters` steps, loss history [iters + 1] of
    L(beta^t) + lam |beta^t|_1)."""
    K = np.asarray(K, dtype=np.float64)
    a = np.asarray(alpha, dtype=np.float64)
    b = np.array(beta0, dtype=np.float64)
    hist = []
    for _ in range(iters):
        r = a - b
        g = K @ r
        hist.append(float(r @ g) + lam * float(np.abs(b).sum()))
        b = soft_threshold(b + 2.0 * gamma * g, gamma * lam)
    r = a - b
    hist.append(float(r @ (K @ r)) + lam * float(np.abs(b).sum()))
    return b, np.array(hist)
