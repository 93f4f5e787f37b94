"""Pins the FP64 oracle to facts fixed by the paper and by mathematics.

Each test would fail under a plausible slip in the oracle: a dropped 1/2 or
4^-lambda, a swapped index (p vs q, L vs M), a wrong boundary value, a sign
error in the stencil, or a mis-derived adjoint.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2006_14794_gb300 import inputs
from tests import truth


# ---------------------------------------------------------------- closed forms
# of the DISCRETE scheme (Sec. 3.1, explicit scheme on P_lambda), derived by hand.

def _two_point(v):
    return np.array([np.zeros_like(v), v])


def test_single_cell_lambda0():
    # One coarse cell, P_0: k(1,1) = 1 + 1 - 1 + 1/2 G (1 + 1) = 1 + G.
    x = _two_point(np.array([0.7, -0.2, 0.1]))
    y = _two_point(np.array([0.4, 0.9, -1.3]))
    G = float(np.dot(x[1], y[1]))
    assert oracle.sigkernel(x, y, 0) == pytest.approx(1.0 + G, rel=1e-15)


def test_single_cell_lambda1():
    # One coarse cell refined 2x2, g = G/4 per refined cell:
    # k(1,1)=1+g, k(1,2)=k(2,1)=1+2g+g^2/2, k(2,2)=1+4g+3g^2+g^3/2
    # = 1 + G + 3G^2/16 + G^3/128.
    x = _two_point(np.array([1.0, 0.5]))
    y = _two_point(np.array([0.3, 2.0]))
    G = 1.3
    want = 1 + G + 3 * G ** 2 / 16 + G ** 3 / 128
    assert oracle.sigkernel(x, y, 1) == pytest.approx(want, rel=1e-15)


@pytest.mark.parametrize("transpose", [False, True])
def test_one_row_product_form(transpose):
    # x has one increment, y has n: the single refined row obeys
    # k(1,b) + 1 = (1 + g_b/2) (k(1,b-1) + 1), so k = 2 prod_b (1 + g_b/2) - 1.
    rng = np.random.default_rng(5)
    x = _two_point(rng.normal(size=3))
    y = np.cumsum(np.vstack([np.zeros(3), rng.normal(size=(6, 3))]), axis=0)
    g = np.diff(y, axis=0) @ (x[1] - x[0])
    want = 2.0 * np.prod(1.0 + g / 2.0) - 1.0
    got = oracle.sigkernel(y, x, 0) if transpose else oracle.sigkernel(x, y, 0)
    assert got == pytest.approx(want, rel=1e-14)


def test_one_row_refined_equals_subdivided_points():
    # The remark after the scheme: refining P_0 by 2^lambda is the same as
    # inserting the 2^lambda - 1 midpoints of every linear segment.
    rng = np.random.default_rng(6)
    x = np.cumsum(rng.normal(size=(5, 2)) * 0.4, axis=0)
    y = np.cumsum(rng.normal(size=(4, 2)) * 0.4, axis=0)

    def subdivide(p, s):
        out = [p[0]]
        for i in range(len(p) - 1):
            for k in range(1, s + 1):
                out.append(p[i] + (p[i + 1] - p[i]) * k / s)
        return np.array(out)

    for lam in (1, 2):
        s = 2 ** lam
        a = oracle.sigkernel(x, y, lam)
        b = oracle.sigkernel(subdivide(x, s), subdivide(y, s), 0)
        assert a == pytest.approx(b, rel=1e-13)


# ---------------------------------------------- convergence to the true kernel
# (global error theorem, Sec. 3.1: |k - k_lambda| <= K 4^-lambda)

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_straight_lines_converge_to_bessel(seed):
    # x = a t, y = b t: constant <x', y'> = <a,b>, whose Goursat solution is the
    # Riemann function I_0(2 sqrt(<a,b> s t)) (Appendix A, sigma = tau = 1).
    rng = np.random.default_rng(seed)
    a, b = rng.normal(0, np.sqrt(1 / 3), 3), rng.normal(0, np.sqrt(1 / 3), 3)
    t = np.linspace(0, 1, 9)[:, None]
    x, y = a * t, b * t
    true = truth.series_I0(float(a @ b))
    ks = [oracle.sigkernel(x, y, lam) for lam in range(0, 7)]
    errs = [abs(k - true) for k in ks]
    for e0, e1 in zip(errs[2:-1], errs[3:]):
        assert 3.5 < e0 / e1 < 4.5
    assert truth.richardson(ks[5], ks[6]) == pytest.approx(true, rel=1e-8)


def test_one_dimensional_paths_closed_form():
    # d = 1: S(x) = exp(x_T - x_0) (Thm. "universal", commutative case), so
    # k = sum_k (dX dY)^k / (k!)^2 for ANY 1-D path.
    rng = np.random.default_rng(11)
    x = np.cumsum(rng.normal(size=(7, 1)) * 0.5, axis=0)
    y = np.cumsum(rng.normal(size=(5, 1)) * 0.5, axis=0)
    true = truth.series_I0(float((x[-1, 0] - x[0, 0]) * (y[-1, 0] - y[0, 0])))
    k5, k6 = oracle.sigkernel(x, y, 5), oracle.sigkernel(x, y, 6)
    assert truth.richardson(k5, k6) == pytest.approx(true, rel=1e-7)
    assert abs(oracle.sigkernel(x, y, 2) - true) > 4 * abs(k6 - true)


@pytest.mark.parametrize("seed,d,L,M", [(21, 2, 3, 4), (22, 3, 4, 3), (23, 2, 5, 2)])
def test_brute_force_truncated_signatures(seed, d, L, M):
    # k = <S(x), S(y)> (definition of the signature kernel), brute force.
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.normal(size=(L, d)) * 0.35, axis=0)
    y = np.cumsum(rng.normal(size=(M, d)) * 0.35, axis=0)
    true, tail = truth.sig_inner(x, y, 12)
    assert tail < 1e-10
    k6, k7 = oracle.sigkernel(x, y, 6), oracle.sigkernel(x, y, 7)
    assert truth.richardson(k6, k7) == pytest.approx(true, abs=2e-8 + tail)


# -------------------------------------------------------------------- invariants

def test_symmetry_bitwise():
    X = inputs.random_paths(31, 4, 17, 3, time_channel=True)
    Y = inputs.random_paths(32, 4, 11, 3, time_channel=True)
    for lam in (0, 1, 2):
        for i in range(4):
            assert oracle.sigkernel(X[i], Y[i], lam) == oracle.sigkernel(Y[i], X[i], lam)


def test_repeated_points_invariance():
    rng = np.random.default_rng(41)
    x = np.cumsum(rng.normal(size=(8, 3)) * 0.3, axis=0)
    y = np.cumsum(rng.normal(size=(6, 3)) * 0.3, axis=0)
    x_rep = np.insert(x, 3, x[3], axis=0)     # zero increment
    y_rep = np.insert(y, 0, y[0], axis=0)
    for lam in (0, 1, 2):
        k = oracle.sigkernel(x, y, lam)
        assert oracle.sigkernel(x_rep, y_rep, lam) == pytest.approx(k, rel=1e-14)


def test_trivial_cases_are_exactly_one():
    rng = np.random.default_rng(42)
    x = np.cumsum(rng.normal(size=(9, 4)), axis=0)
    const = np.repeat(rng.normal(size=(1, 4)), 7, axis=0)
    assert oracle.sigkernel(x, const, 2) == 1.0
    xo = np.zeros((9, 4)); xo[:, :2] = x[:, :2]
    yo = np.zeros((6, 4)); yo[:, 2:] = np.cumsum(rng.normal(size=(6, 2)), axis=0)
    assert oracle.sigkernel(xo, yo, 1) == 1.0
    assert oracle.sigkernel(x[:1], x, 1) == 1.0


def test_scaling_and_rotation():
    rng = np.random.default_rng(43)
    x = np.cumsum(rng.normal(size=(10, 3)) * 0.3, axis=0)
    y = np.cumsum(rng.normal(size=(12, 3)) * 0.3, axis=0)
    assert oracle.sigkernel(1.7 * x, y, 1) == pytest.approx(oracle.sigkernel(x, 1.7 * y, 1), rel=1e-14)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    assert oracle.sigkernel(x @ Q, y @ Q, 2) == pytest.approx(oracle.sigkernel(x, y, 2), rel=1e-12)


def test_batched_entry_points_agree_with_single_pair():
    X = inputs.random_paths(51, 3, 9, 2)
    Y = inputs.random_paths(52, 4, 7, 2)
    G = oracle.gram(X, Y, 1)
    for i in range(3):
        for j in range(4):
            assert G[i, j] == oracle.sigkernel(X[i], Y[j], 1)
    P = oracle.pairs(X, Y[:3], 2)
    assert all(P[i] == oracle.sigkernel(X[i], Y[i], 2) for i in range(3))
    xo = np.array([0, 9, 14, 23]); yo = np.array([0, 7, 11, 18])
    Xp = np.concatenate([X[0], X[1][:5], X[2]]); Yp = np.concatenate([Y[0], Y[1][:4], Y[2]])
    V = oracle.pairs_varlen(Xp, xo, Yp, yo, 1)
    assert V[1] == oracle.sigkernel(X[1][:5], Y[1][:4], 1)
    assert V[2] == oracle.sigkernel(X[2], Y[2], 1)


# ---------------------------------------------------------------------- gradient
# (reverse mode of the discrete scheme; the paper states no gradient)

def test_gradient_matches_hand_derivative():
    # single coarse cell, lambda = 1: k = 1 + G + 3G^2/16 + G^3/128,
    # dk/dx_1 = k'(G) dy, dk/dx_0 = -k'(G) dy.
    x = _two_point(np.array([1.0, 0.5]))
    y = _two_point(np.array([0.3, 2.0]))
    G = 1.3
    kp = 1 + 3 * G / 8 + 3 * G ** 2 / 128
    k, dx, dy = oracle.sigkernel_grad(x, y, 1)
    np.testing.assert_allclose(dx[1], kp * y[1], rtol=1e-14)
    np.testing.assert_allclose(dx[0], -kp * y[1], rtol=1e-14)
    np.testing.assert_allclose(dy[1], kp * x[1], rtol=1e-14)


def _fd4(f, arr, idx, h=1e-3):
    """Fourth-order central difference (the h^2 term cancelled)."""
    def at(t):
        a = arr.copy()
        a[idx] += t
        return f(a)
    return (8 * (at(h) - at(-h)) - (at(2 * h) - at(-2 * h))) / (12 * h)


@pytest.mark.parametrize("lam", [0, 1, 2])
def test_gradient_matches_central_differences(lam):
    # A fourth-order stencil at h = 1e-3: the plain h = 1e-6 difference carries
    # ~1e-9 of rounding noise, more than the adjoint's own error.
    rng = np.random.default_rng(60 + lam)
    x = np.cumsum(rng.normal(size=(6, 3)) * 0.3, axis=0)
    y = np.cumsum(rng.normal(size=(5, 3)) * 0.3, axis=0)
    k, dx, dy = oracle.sigkernel_grad(x, y, lam)
    assert k == oracle.sigkernel(x, y, lam)
    for idx in np.ndindex(x.shape):
        fd = _fd4(lambda a: oracle.sigkernel(a, y, lam), x, idx)
        assert dx[idx] == pytest.approx(fd, rel=1e-9, abs=1e-11)
    for idx in np.ndindex(y.shape):
        fd = _fd4(lambda a: oracle.sigkernel(x, a, lam), y, idx)
        assert dy[idx] == pytest.approx(fd, rel=1e-9, abs=1e-11)


def test_batched_gradients_agree_with_single_pair():
    X = inputs.random_paths(71, 3, 6, 2)
    Y = inputs.random_paths(72, 2, 5, 2)
    gout = np.array([[0.3, -1.2], [0.7, 0.1], [-0.4, 2.0]])
    dX, dY = oracle.gram_grad(X, Y, 1, gout)
    for i in range(3):
        want = sum(gout[i, j] * oracle.sigkernel_grad(X[i], Y[j], 1)[1] for j in range(2))
        np.testing.assert_allclose(dX[i], want, rtol=1e-13, atol=1e-15)
    for j in range(2):
        want = sum(gout[i, j] * oracle.sigkernel_grad(X[i], Y[j], 1)[2] for i in range(3))
        np.testing.assert_allclose(dY[j], want, rtol=1e-13, atol=1e-15)
    g = np.array([0.5, -1.5])
    pX, pY = oracle.pairs_grad(X[:2], Y, 2, g)
    for b in range(2):
        _, dx, dy = oracle.sigkernel_grad(X[b], Y[b], 2, g[b])
        np.testing.assert_allclose(pX[b], dx, rtol=1e-14)
        np.testing.assert_allclose(pY[b], dy, rtol=1e-14)


# --------------------------------------------------------------------------- MMD

def test_mmd_constant_paths_is_zero():
    X = np.repeat(np.random.default_rng(80).normal(size=(5, 1, 3)), 6, axis=1)
    Y = np.repeat(np.random.default_rng(81).normal(size=(4, 1, 3)), 6, axis=1)
    assert oracle.mmd2(X, Y, 1) == 0.0


def test_mmd_orthogonal_batches():
    # Cross terms are exactly 1 when X and Y live in orthogonal channels, so
    # MMD^2 = mean off-diagonal k(x_i,x_j) + mean off-diagonal k(y_i,y_j) - 2.
    X = inputs.random_paths(82, 5, 8, 4, scale=2.0); X[:, :, 2:] = 0
    Y = inputs.random_paths(83, 4, 8, 4, scale=2.0); Y[:, :, :2] = 0
    kx = [oracle.sigkernel(X[i], X[j], 1) for i in range(5) for j in range(5) if i != j]
    ky = [oracle.sigkernel(Y[i], Y[j], 1) for i in range(4) for j in range(4) if i != j]
    assert oracle.mmd2(X, Y, 1) == pytest.approx(np.mean(kx) + np.mean(ky) - 2.0, rel=1e-13)


def test_mmd_is_unbiased_under_the_null():
    # E[MMD^2_u] = 0 when both batches come from the same law.
    vals = []
    for r in range(40):
        Z = inputs.random_paths(1000 + r, 12, 10, 2, scale=3.0)
        vals.append(oracle.mmd2(Z[:6], Z[6:], 0))
    vals = np.array(vals)
    assert abs(vals.mean()) < 3.0 * vals.std() / np.sqrt(len(vals)) + 1e-12


def test_mmd_gradient_matches_central_differences():
    X = inputs.random_paths(90, 3, 5, 2, scale=2.0)
    Y = inputs.random_paths(91, 3, 5, 2, scale=2.0)
    g = oracle.mmd2_grad_x(X, Y, 1)
    for idx in [(0, 1, 0), (1, 4, 1), (2, 2, 0), (0, 0, 1)]:
        fd = _fd4(lambda a: oracle.mmd2(a, Y, 1), X, idx)
        assert g[idx] == pytest.approx(fd, rel=1e-8, abs=1e-11)
