"""Pins the oracle's two variants of the scheme to facts fixed by the paper and
by mathematics:

* the implicit scheme of the remark after the explicit one (Sec. 3.1), whose
  quadrature uses all four corner values;
* the static-kernel lift (Sec. 2.2): the PDE of the paths mapped into a
  feature space by a static kernel, here the RBF kernel, whose coefficient on a
  coarse cell is the second difference of kappa over the cell's corners.

Each test would fail under a plausible slip: a weight 1/4 taken as 1/2, the
unknown corner dropped from the quadrature, a sign or corner of the second
difference swapped, sigma squared twice or not at all, a wrong derivative.
"""
import math

import numpy as np
import pytest

import oracle
from tests import truth


def _two_point(v):
    return np.array([np.zeros_like(v), v])


def _fd4(f, arr, idx, h=1e-3):
    def at(t):
        a = arr.copy()
        a[idx] += t
        return f(a)
    return (8 * (at(h) - at(-h)) - (at(2 * h) - at(-2 * h))) / (12 * h)


# ---------------------------------------------------------- the implicit scheme

def test_implicit_single_cell():
    # One coarse cell on P_0: k (1 - G/4) = 1 + 1 - 1 + G/4 (1 + 1 + 1), so
    # k = (1 + 3G/4) / (1 - G/4).
    x = _two_point(np.array([0.7, -0.2, 0.1]))
    y = _two_point(np.array([0.9, 0.4, 1.3]))
    G = float(np.dot(x[1], y[1]))
    want = (1 + 0.75 * G) / (1 - 0.25 * G)
    assert oracle.sigkernel(x, y, 0, scheme="implicit") == pytest.approx(want, rel=1e-15)
    assert abs(want - (1 + G)) > 1e-3   # differs from the explicit scheme's 1 + G


@pytest.mark.parametrize("transpose", [False, True])
def test_implicit_one_row_product_form(transpose):
    # One refined row: k_b (1 - g_b/4) = k_{b-1} (1 + g_b/4) + g_b/2, i.e.
    # (k_b + 1)(1 - g_b/4) = (k_{b-1} + 1)(1 + g_b/4), so
    # k = 2 prod_b (1 + g_b/4) / (1 - g_b/4) - 1.
    rng = np.random.default_rng(105)
    x = _two_point(rng.normal(size=3))
    y = np.cumsum(np.vstack([np.zeros(3), rng.normal(size=(6, 3))]), axis=0)
    g = np.diff(y, axis=0) @ (x[1] - x[0])
    want = 2.0 * np.prod((1.0 + g / 4.0) / (1.0 - g / 4.0)) - 1.0
    got = (oracle.sigkernel(y, x, 0, scheme="implicit") if transpose
           else oracle.sigkernel(x, y, 0, scheme="implicit"))
    assert got == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("seed", [0, 1])
def test_implicit_converges_to_bessel(seed):
    # Straight lines x = a t, y = b t: the Goursat solution is the Riemann
    # function I_0(2 sqrt(<a,b>)) (Appendix A).  The trapezoidal quadrature of
    # the implicit scheme is second order too: the error falls ~4x per level.
    rng = np.random.default_rng(seed)
    a, b = rng.normal(0, np.sqrt(1 / 3), 3), rng.normal(0, np.sqrt(1 / 3), 3)
    t = np.linspace(0, 1, 9)[:, None]
    x, y = a * t, b * t
    true = truth.series_I0(float(a @ b))
    ks = [oracle.sigkernel(x, y, lam, scheme="implicit") for lam in range(0, 7)]
    errs = [abs(k - true) for k in ks]
    for e0, e1 in zip(errs[2:-1], errs[3:]):
        assert 3.5 < e0 / e1 < 4.5
    assert truth.richardson(ks[5], ks[6]) == pytest.approx(true, rel=1e-8)
    # the two schemes differ at a given level and meet in the limit
    ke = [oracle.sigkernel(x, y, lam) for lam in (1, 6)]
    assert abs(ke[0] - ks[1]) > 10 * abs(ke[1] - ks[6])


def test_implicit_brute_force_truncated_signatures():
    rng = np.random.default_rng(123)
    x = np.cumsum(rng.normal(size=(4, 2)) * 0.35, axis=0)
    y = np.cumsum(rng.normal(size=(3, 2)) * 0.35, axis=0)
    true, tail = truth.sig_inner(x, y, 12)
    k6 = oracle.sigkernel(x, y, 6, scheme="implicit")
    k7 = oracle.sigkernel(x, y, 7, scheme="implicit")
    assert truth.richardson(k6, k7) == pytest.approx(true, abs=2e-8 + tail)


def test_implicit_symmetry_and_trivial_cases():
    rng = np.random.default_rng(124)
    x = np.cumsum(rng.normal(size=(7, 3)) * 0.3, axis=0)
    y = np.cumsum(rng.normal(size=(5, 3)) * 0.3, axis=0)
    for lam in (0, 2):
        assert oracle.sigkernel(x, y, lam, scheme="implicit") == pytest.approx(
            oracle.sigkernel(y, x, lam, scheme="implicit"), rel=1e-14)
    z = np.zeros((5, 3))
    z[:, 0] = 1.0
    w = np.zeros((4, 3))
    w[:, 1] = np.linspace(0, 2, 4)
    assert oracle.sigkernel(z, y, 1, scheme="implicit") == 1.0   # constant path
    assert oracle.sigkernel(np.cumsum(z, axis=0) * [1, 0, 0], w, 1, scheme="implicit") == 1.0


def test_implicit_single_cell_gradient():
    # k = (1 + 3G/4)/(1 - G/4): dk/dG = 1/(1 - G/4)^2; G = <x1 - x0, y1 - y0>.
    x = _two_point(np.array([0.7, -0.2, 0.1]))
    y = _two_point(np.array([0.4, 0.9, -1.3]))
    G = float(np.dot(x[1], y[1]))
    dkdG = 1.0 / (1 - 0.25 * G) ** 2
    k, dx, dy = oracle.sigkernel_grad(x, y, 0, scheme="implicit")
    np.testing.assert_allclose(dx, dkdG * np.array([-y[1], y[1]]), rtol=1e-14)
    np.testing.assert_allclose(dy, dkdG * np.array([-x[1], x[1]]), rtol=1e-14)


@pytest.mark.parametrize("lam", [0, 1])
def test_implicit_gradient_matches_central_differences(lam):
    rng = np.random.default_rng(160 + lam)
    x = np.cumsum(rng.normal(size=(6, 3)) * 0.3, axis=0)
    y = np.cumsum(rng.normal(size=(5, 3)) * 0.3, axis=0)
    k, dx, dy = oracle.sigkernel_grad(x, y, lam, scheme="implicit")
    assert k == oracle.sigkernel(x, y, lam, scheme="implicit")
    for idx in np.ndindex(x.shape):
        fd = _fd4(lambda a: oracle.sigkernel(a, y, lam, scheme="implicit"), x, idx)
        assert dx[idx] == pytest.approx(fd, rel=1e-9, abs=1e-11)
    for idx in np.ndindex(y.shape):
        fd = _fd4(lambda a: oracle.sigkernel(x, a, lam, scheme="implicit"), y, idx)
        assert dy[idx] == pytest.approx(fd, rel=1e-9, abs=1e-11)


# ------------------------------------------------------------ the RBF lift

def _rbf_features_1d(a, sigma, N):
    # exp(-(a-b)^2 / 2 s^2) = e^{-a^2/2s^2} e^{-b^2/2s^2} sum_n (ab/s^2)^n / n!:
    # phi_n(a) = e^{-a^2/2s^2} (a/s)^n / sqrt(n!), n = 0..N
    n = np.arange(N + 1)
    lf = np.array([math.lgamma(k + 1) for k in n])
    return np.exp(-a[:, None] ** 2 / (2 * sigma ** 2)) * (a[:, None] / sigma) ** n / np.exp(lf / 2)


def _rbf_lift(path, sigma, N=40):
    # product kernel over channels: phi(a) = phi(a_1) (x) ... (x) phi(a_d)
    out = _rbf_features_1d(path[:, 0], sigma, N)
    for c in range(1, path.shape[1]):
        f = _rbf_features_1d(path[:, c], sigma, N)
        out = (out[:, :, None] * f[:, None, :]).reshape(path.shape[0], -1)
    return out


@pytest.mark.parametrize("d,lam,scheme", [(1, 0, "explicit"), (1, 2, "explicit"),
                                          (2, 1, "explicit"), (2, 1, "implicit")])
def test_rbf_equals_linear_kernel_of_lifted_paths(d, lam, scheme):
    # Sec. 2.2: the lifted PDE is the PDE of the paths phi(x), phi(y) in the
    # feature space.  With an explicit (truncated Taylor) feature map of the
    # RBF kernel, the linear-kernel oracle on the lifted points must give the
    # RBF-lifted value: the second difference of kappa is exactly
    # <phi(x_{p+1}) - phi(x_p), phi(y_{q+1}) - phi(y_q)> by bilinearity.
    rng = np.random.default_rng(200 + d + lam)
    x = np.cumsum(rng.normal(size=(5, d)) * 0.4, axis=0)
    y = np.cumsum(rng.normal(size=(4, d)) * 0.4, axis=0)
    sigma = 0.8
    want = oracle.sigkernel(_rbf_lift(x, sigma), _rbf_lift(y, sigma), lam, scheme=scheme)
    got = oracle.sigkernel(x, y, lam, scheme=scheme, static_kernel="rbf", sigma=sigma)
    assert got == pytest.approx(want, rel=1e-13)
    # and the lift is not the identity: the linear kernel of x, y differs
    assert abs(got - oracle.sigkernel(x, y, lam, scheme=scheme)) > 1e-3


def test_rbf_single_cell_special_point():
    # x = y = (0, u) in one channel with u^2 / (2 sigma^2) = ln 2:
    # G = k(u,u) - k(0,u) - k(u,0) + k(0,0) = 1 - 1/2 - 1/2 + 1 = 1, so
    # k = 1 + G = 2 on P_0 and 1 + G + 3G^2/16 + G^3/128 on P_1.
    sigma = 1.0
    u = math.sqrt(2 * math.log(2.0)) * sigma
    x = np.array([[0.0], [u]])
    assert oracle.sigkernel(x, x, 0, static_kernel="rbf", sigma=sigma) == pytest.approx(2.0, rel=1e-15)
    assert oracle.sigkernel(x, x, 1, static_kernel="rbf", sigma=sigma) == pytest.approx(
        2.0 + 3.0 / 16 + 1.0 / 128, rel=1e-15)


def test_rbf_invariances():
    # Only |x_p - y_q| enters: a common translation or rotation of both paths
    # leaves k unchanged; translating one path alone does not.
    rng = np.random.default_rng(210)
    x = np.cumsum(rng.normal(size=(6, 3)) * 0.4, axis=0)
    y = np.cumsum(rng.normal(size=(5, 3)) * 0.4, axis=0)
    v = rng.normal(size=3)
    Qm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    k = oracle.sigkernel(x, y, 1, static_kernel="rbf", sigma=0.7)
    assert oracle.sigkernel(x + v, y + v, 1, static_kernel="rbf", sigma=0.7) == pytest.approx(k, rel=1e-13)
    assert oracle.sigkernel(x @ Qm.T, y @ Qm.T, 1, static_kernel="rbf", sigma=0.7) == pytest.approx(
        k, rel=1e-13)
    assert abs(oracle.sigkernel(x + v, y, 1, static_kernel="rbf", sigma=0.7) - k) > 1e-4
    assert oracle.sigkernel(x, y, 1, static_kernel="rbf", sigma=0.7) == pytest.approx(
        oracle.sigkernel(y, x, 1, static_kernel="rbf", sigma=0.7), rel=1e-14)
    const = np.ones((4, 3))
    assert oracle.sigkernel(const, y, 2, static_kernel="rbf", sigma=0.7) == 1.0


def test_rbf_wide_bandwidth_limit():
    # kappa = 1 - |a-b|^2 / (2 s^2) + O(s^-4): the second difference of
    # -|a-b|^2 / (2 s^2) is <dx, dy> / s^2, so the RBF lift of (x, y) tends to
    # the linear kernel of (x/s, y/s) with an error O(s^-4) per cell.
    rng = np.random.default_rng(211)
    x = np.cumsum(rng.normal(size=(6, 2)) * 0.5, axis=0)
    y = np.cumsum(rng.normal(size=(5, 2)) * 0.5, axis=0)
    diffs = []
    for s in (0.5, 1.0, 2.0):
        s_eff = s * 4.0
        diffs.append(abs(oracle.sigkernel(x, y, 1, static_kernel="rbf", sigma=s_eff)
                         - oracle.sigkernel(x / s_eff, y / s_eff, 1)))
    for a, b in zip(diffs, diffs[1:]):
        assert 10 < a / b < 20   # doubling sigma: error / 16 (O(s^-4))


@pytest.mark.parametrize("scheme", ["explicit", "implicit"])
def test_rbf_gradient_matches_central_differences(scheme):
    rng = np.random.default_rng(220)
    x = np.cumsum(rng.normal(size=(5, 2)) * 0.4, axis=0)
    y = np.cumsum(rng.normal(size=(4, 2)) * 0.4, axis=0)
    kw = dict(scheme=scheme, static_kernel="rbf", sigma=0.6)
    k, dx, dy = oracle.sigkernel_grad(x, y, 1, **kw)
    assert k == oracle.sigkernel(x, y, 1, **kw)
    for idx in np.ndindex(x.shape):
        fd = _fd4(lambda a: oracle.sigkernel(a, y, 1, **kw), x, idx)
        assert dx[idx] == pytest.approx(fd, rel=1e-8, abs=1e-11)
    for idx in np.ndindex(y.shape):
        fd = _fd4(lambda a: oracle.sigkernel(x, a, 1, **kw), y, idx)
        assert dy[idx] == pytest.approx(fd, rel=1e-8, abs=1e-11)


def test_variant_batched_entry_points_agree_with_single_pair():
    rng = np.random.default_rng(230)
    X = np.cumsum(rng.normal(size=(3, 6, 2)) * 0.3, axis=1)
    Y = np.cumsum(rng.normal(size=(2, 5, 2)) * 0.3, axis=1)
    for kw in (dict(scheme="implicit"), dict(static_kernel="rbf", sigma=0.9),
               dict(scheme="implicit", static_kernel="rbf", sigma=1.3)):
        G = oracle.gram(X, Y, 1, **kw)
        for i in range(3):
            for j in range(2):
                assert G[i, j] == oracle.sigkernel(X[i], Y[j], 1, **kw)
        P = oracle.pairs(X[:2], Y, 1, **kw)
        assert P[1] == oracle.sigkernel(X[1], Y[1], 1, **kw)
        xo = np.array([0, 6, 12])
        yo = np.array([0, 5, 10])
        V = oracle.pairs_varlen(X[:2].reshape(-1, 2), xo, Y.reshape(-1, 2), yo, 1, **kw)
        np.testing.assert_array_equal(V, P)
        gout = np.array([[0.3, -1.2], [0.7, 0.1], [-0.4, 2.0]])
        dX, dY = oracle.gram_grad(X, Y, 1, gout, **kw)
        want = sum(gout[0, j] * oracle.sigkernel_grad(X[0], Y[j], 1, **kw)[1] for j in range(2))
        np.testing.assert_allclose(dX[0], want, rtol=1e-13, atol=1e-15)
        pX, pY = oracle.pairs_grad(X[:2], Y, 1, np.array([0.5, -1.5]), **kw)
        _, dx, dy = oracle.sigkernel_grad(X[1], Y[1], 1, -1.5, **kw)
        np.testing.assert_allclose(pY[1], dy, rtol=1e-14)
    with pytest.raises(ValueError):
        oracle.sigkernel(X[0], Y[0], 0, static_kernel="rbf", sigma=0.0)


# ------------------------------------------------------- the solution surface

@pytest.mark.parametrize("lam,kw", [(0, {}), (2, {}), (1, dict(scheme="implicit")),
                                    (1, dict(static_kernel="rbf", sigma=0.7))])
def test_surface_is_the_kernel_of_truncated_paths(lam, kw):
    # The solution at (s_i, t_j) solves the same Goursat problem on the
    # sub-rectangle [u, s_i] x [v, t_j] (Thm. "PDE" on the restricted paths),
    # and the scheme restricted to the sub-grid is the same arithmetic: the
    # surface equals the kernel of the paths cut after their i-th and j-th points.
    rng = np.random.default_rng(300 + lam)
    x = np.cumsum(rng.normal(size=(6, 3)) * 0.4, axis=0)
    y = np.cumsum(rng.normal(size=(5, 3)) * 0.4, axis=0)
    surf = oracle.surface(x, y, lam, **kw)
    assert surf.shape == (6, 5)
    assert np.all(surf[0, :] == 1.0) and np.all(surf[:, 0] == 1.0)
    for i in range(1, 6):
        for j in range(1, 5):
            assert surf[i, j] == oracle.sigkernel(x[:i + 1], y[:j + 1], lam, **kw)
    k, S = oracle.pairs_surface(x[None], y[None], lam, **kw)
    np.testing.assert_array_equal(S[0], surf)
    assert k[0] == surf[-1, -1]


def test_surface_converges_to_bessel_at_every_node():
    # straight lines x = a t, y = b t on [0, 1]: k(s, t) = I_0(2 sqrt(<a,b> s t))
    # (Appendix A); every node's error falls ~4x per dyadic level.
    rng = np.random.default_rng(310)
    a, b = rng.normal(0, np.sqrt(1 / 3), 3), rng.normal(0, np.sqrt(1 / 3), 3)
    t = np.linspace(0, 1, 5)[:, None]
    x, y = a * t, b * t
    ab = float(a @ b)
    true = np.array([[truth.series_I0(ab * si * tj) for tj in t[:, 0]] for si in t[:, 0]])
    errs = [np.abs(oracle.surface(x, y, lam) - true)[1:, 1:] for lam in (3, 4, 5)]
    for e0, e1 in zip(errs, errs[1:]):
        ratio = e0[e0 > 1e-12] / e1[e0 > 1e-12]
        assert np.all((ratio > 3.5) & (ratio < 4.5))
