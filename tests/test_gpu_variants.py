"""The scheme variants through the C ABI against the FP64 oracle: the implicit
four-point scheme of the remark after the explicit scheme (Sec. 3.1), on every
schedule (chained, band, strip with each coefficient kernel, plain; f32 and
f64; uniform and uneven lengths), forward and backward."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
F64_TOL = 1e-11
GRAD_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    from paper_2006_14794_gb300 import sigk
    sigk.lib()


def S():
    from paper_2006_14794_gb300 import sigk
    return sigk


def implicit():
    return S().Variant(scheme="implicit")


def grad_err(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30))


# (rec, rows_per_lane, coef_path, lam, L, M, d): one case per schedule family
FORWARD_CASES = [
    ("chain", 16, 0, 2, 128, 128, 8),     # the bench kernel's instance
    ("chain", 8, 0, 1, 100, 90, 4),
    ("band", 16, 0, 1, 256, 256, 32),     # the MMD shape
    ("band", 8, 3, 0, 230, 256, 40),      # band coefficients on tcgen05
    ("strip", 16, 1, 1, 300, 700, 16),    # FMA coefficients
    ("strip", 8, 2, 2, 150, 90, 40),      # mma.sync coefficients
    ("strip", 4, 3, 1, 200, 260, 64),     # tcgen05 coefficients
    ("plain", 0, 0, 1, 60, 75, 5),
]


@pytest.mark.parametrize("rec,R,coef,lam,L,M,d", FORWARD_CASES)
def test_implicit_forward_matches_oracle(rec, R, coef, lam, L, M, d):
    sigk = S()
    recs = {"chain": sigk.REC_CHAIN, "band": sigk.REC_BAND, "strip": sigk.REC_STRIP,
            "plain": sigk.REC_PLAIN}
    Bx, By = 5, 6
    # unit-scale walks keep every kernel value well away from 0, where the
    # FP32 grid's absolute rounding (values up to ~10 at larger scales) would
    # dominate the relative error of a small corner value
    X32, X64 = inputs.f32(inputs.random_paths(5100 + lam + d, Bx, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(5200 + lam + d, By, M, d, time_channel=True))
    ref = oracle.gram(X64, Y64, lam, scheme="implicit")
    s = sigk.Schedule(recs[rec], R, coef)
    got = sigk.gram(to_dev(X32), to_dev(Y32), lam, schedule=s, variant=implicit(),
                    check_status=True).cpu().numpy()
    assert rel_err(got, ref) <= F32_TOL
    # the variant is really applied: the explicit scheme differs by far more
    assert rel_err(oracle.gram(X64, Y64, lam), ref) > 10 * F32_TOL


@pytest.mark.parametrize("rec", ["strip", "plain"])
def test_implicit_forward_f64(rec):
    sigk = S()
    lam, d = 1, 6
    X = inputs.random_paths(5300, 4, 70, d, scale=2.0, time_channel=True)
    Y = inputs.random_paths(5301, 3, 90, d, scale=2.0, time_channel=True)
    ref = oracle.gram(X, Y, lam, scheme="implicit")
    r = sigk.REC_STRIP if rec == "strip" else sigk.REC_PLAIN
    got = sigk.gram(to_dev(X, torch.float64), to_dev(Y, torch.float64), lam, rec=r,
                    variant=implicit(), check_status=True).cpu().numpy()
    assert rel_err(got, ref) <= F64_TOL


def test_implicit_varlen_matches_oracle():
    sigk = S()
    rng = np.random.default_rng(54)
    lx = rng.integers(2, 200, size=30)
    ly = rng.integers(2, 200, size=30)
    d, lam = 16, 1
    Xp = np.concatenate([inputs.random_paths(5400 + i, 1, int(n), d, scale=2.0)[0] for i, n in enumerate(lx)])
    Yp = np.concatenate([inputs.random_paths(5500 + i, 1, int(n), d, scale=2.0)[0] for i, n in enumerate(ly)])
    xo = np.concatenate([[0], np.cumsum(lx)]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(ly)]).astype(np.int64)
    X32, X64 = inputs.f32(Xp)
    Y32, Y64 = inputs.f32(Yp)
    ref = oracle.pairs_varlen(X64, xo, Y64, yo, lam, scheme="implicit")
    got = sigk.pairs_varlen(to_dev(X32), torch.as_tensor(xo).cuda(), to_dev(Y32),
                            torch.as_tensor(yo).cuda(), lam, int(max(lx.max(), ly.max())),
                            variant=implicit(), check_status=True).cpu().numpy()
    assert rel_err(got, ref) <= F32_TOL


@pytest.mark.parametrize("rec,dtype", [("band", torch.float32), ("strip", torch.float32),
                                       ("plain", torch.float32), ("plain", torch.float64),
                                       ("strip", torch.float64)])
def test_implicit_gram_backward_matches_oracle(rec, dtype):
    sigk = S()
    recs = {"band": sigk.REC_BAND, "strip": sigk.REC_STRIP, "plain": sigk.REC_PLAIN}
    lam, d, L, M = 1, 12, 60, 45
    Bx, By = 4, 3
    X32, X64 = inputs.f32(inputs.random_paths(5600, Bx, L, d, scale=2.0, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(5601, By, M, d, scale=2.0, time_channel=True))
    gout = np.random.default_rng(56).normal(size=(Bx, By))
    rX, rY = oracle.gram_grad(X64, Y64, lam, gout, scheme="implicit")
    Xd = to_dev(X32 if dtype == torch.float32 else X64, dtype)
    Yd = to_dev(Y32 if dtype == torch.float32 else Y64, dtype)
    dX, dY = sigk.gram_backward(to_dev(gout, dtype), Xd, Yd, lam, rec=recs[rec], variant=implicit())
    tol = GRAD_TOL if dtype == torch.float32 else 1e-10
    assert grad_err(dX.cpu(), rX) <= tol
    assert grad_err(dY.cpu(), rY) <= tol
    # and not the explicit scheme's gradient
    eX, _ = oracle.gram_grad(X64, Y64, lam, gout)
    assert grad_err(eX, rX) > 100 * GRAD_TOL


def test_implicit_symmetric_and_autograd():
    sigk = S()
    lam, d, L, B = 1, 32, 100, 5
    X32, X64 = inputs.f32(inputs.random_paths(5700, B, L, d, time_channel=True))
    gout = np.random.default_rng(57).normal(size=(B, B))
    rX, rY = oracle.gram_grad(X64, X64, lam, gout, scheme="implicit")
    X = to_dev(X32).requires_grad_(True)
    K = sigk.SigKernelGram.apply(X, X, lam, implicit())
    assert rel_err(K.detach().cpu().numpy(), oracle.gram(X64, X64, lam, scheme="implicit")) <= F32_TOL
    K.backward(to_dev(gout))
    assert grad_err(X.grad.cpu(), rX + rY) <= GRAD_TOL
    g = np.random.default_rng(58).normal(size=B)
    Y32, Y64 = inputs.f32(inputs.random_paths(5701, B, 80, d, time_channel=True))
    Xp = to_dev(X32).requires_grad_(True)
    Yp = to_dev(Y32).requires_grad_(True)
    k = sigk.SigKernelPairs.apply(Xp, Yp, lam, implicit())
    k.backward(to_dev(g))
    pX, pY = oracle.pairs_grad(X64, Y64, lam, g, scheme="implicit")
    assert grad_err(Xp.grad.cpu(), pX) <= GRAD_TOL
    assert grad_err(Yp.grad.cpu(), pY) <= GRAD_TOL


def test_implicit_bench_shape_sampled_entries():
    """The 256 x 256 Gram of the benchmark (L = 128, d = 8, dyadic order 2) in
    its launch configuration, checked on sampled entries."""
    sigk = S()
    w = inputs.gram_256()
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    got = sigk.gram(to_dev(X32), to_dev(Y32), 2, variant=implicit()).cpu().numpy()
    rng = np.random.default_rng(59)
    idx = rng.choice(X32.shape[0] * Y32.shape[0], 12, replace=False)
    for t in idx:
        i, j = divmod(int(t), Y32.shape[0])
        ref = oracle.sigkernel(X64[i], Y64[j], 2, scheme="implicit")
        assert rel_err(got[i, j], ref) <= F32_TOL


# ------------------------------------------------------------------ RBF lift

def rbf(sigma, scheme="explicit"):
    return S().Variant(scheme=scheme, static_kernel="rbf", sigma=sigma)


RBF_FORWARD_CASES = [
    # (rec, R, lam, L, M, d, sigma, scheme)
    ("auto", 0, 2, 128, 128, 8, 1.0, "explicit"),   # the bench shape: band form (no inline chain)
    ("band", 16, 1, 256, 256, 32, 2.0, "explicit"),  # the MMD shape
    ("band", 8, 1, 129, 140, 17, 0.7, "implicit"),
    ("band", 4, 0, 100, 120, 5, 0.5, "explicit"),
    ("strip", 16, 1, 300, 700, 16, 1.5, "explicit"),
    ("strip", 8, 2, 150, 90, 40, 3.0, "implicit"),
    ("strip", 4, 1, 200, 260, 64, 4.0, "explicit"),
    ("plain", 0, 1, 60, 75, 5, 0.8, "explicit"),
    ("chain", 0, 1, 40, 50, 3, 0.6, "explicit"),    # CHAIN asked: the band form serves it
]


@pytest.mark.parametrize("rec,R,lam,L,M,d,sigma,scheme", RBF_FORWARD_CASES)
def test_rbf_forward_matches_oracle(rec, R, lam, L, M, d, sigma, scheme):
    sigk = S()
    recs = {"auto": sigk.REC_AUTO, "chain": sigk.REC_CHAIN, "band": sigk.REC_BAND,
            "strip": sigk.REC_STRIP, "plain": sigk.REC_PLAIN}
    Bx, By = 5, 6
    X32, X64 = inputs.f32(inputs.random_paths(6100 + lam + d, Bx, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(6200 + lam + d, By, M, d, time_channel=True))
    v = rbf(sigma, scheme)
    ref = oracle.gram(X64, Y64, lam, scheme=scheme, static_kernel="rbf", sigma=sigma)
    got = sigk.gram(to_dev(X32), to_dev(Y32), lam, schedule=sigk.Schedule(recs[rec], R, 0), variant=v,
                    check_status=True).cpu().numpy()
    assert rel_err(got, ref) <= F32_TOL
    # the lift is applied: the linear kernel differs by far more
    assert rel_err(oracle.gram(X64, Y64, lam, scheme=scheme), ref) > 10 * F32_TOL


@pytest.mark.parametrize("rec", ["strip", "plain"])
def test_rbf_forward_f64(rec):
    sigk = S()
    lam, d, sigma = 1, 6, 0.9
    X = inputs.random_paths(6300, 4, 70, d, time_channel=True)
    Y = inputs.random_paths(6301, 3, 90, d, time_channel=True)
    ref = oracle.gram(X, Y, lam, static_kernel="rbf", sigma=sigma)
    r = sigk.REC_STRIP if rec == "strip" else sigk.REC_PLAIN
    got = sigk.gram(to_dev(X, torch.float64), to_dev(Y, torch.float64), lam, rec=r,
                    variant=rbf(sigma), check_status=True).cpu().numpy()
    assert rel_err(got, ref) <= F64_TOL


def test_rbf_pairs_and_varlen_match_oracle():
    sigk = S()
    lam, d, sigma = 1, 16, 1.2
    X32, X64 = inputs.f32(inputs.random_paths(6400, 40, 90, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(6401, 40, 60, d, time_channel=True))
    ref = oracle.pairs(X64, Y64, lam, static_kernel="rbf", sigma=sigma)
    got = sigk.pairs(to_dev(X32), to_dev(Y32), lam, variant=rbf(sigma)).cpu().numpy()
    assert rel_err(got, ref) <= F32_TOL
    rng = np.random.default_rng(64)
    lx = rng.integers(2, 200, size=30)
    ly = rng.integers(2, 200, size=30)
    Xp = np.concatenate([inputs.random_paths(6500 + i, 1, int(n), d)[0] for i, n in enumerate(lx)])
    Yp = np.concatenate([inputs.random_paths(6600 + i, 1, int(n), d)[0] for i, n in enumerate(ly)])
    xo = np.concatenate([[0], np.cumsum(lx)]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(ly)]).astype(np.int64)
    Xp32, Xp64 = inputs.f32(Xp)
    Yp32, Yp64 = inputs.f32(Yp)
    for scheme in ("explicit", "implicit"):
        ref = oracle.pairs_varlen(Xp64, xo, Yp64, yo, lam, scheme=scheme, static_kernel="rbf", sigma=sigma)
        got = sigk.pairs_varlen(to_dev(Xp32), torch.as_tensor(xo).cuda(), to_dev(Yp32),
                                torch.as_tensor(yo).cuda(), lam, int(max(lx.max(), ly.max())),
                                variant=rbf(sigma, scheme), check_status=True).cpu().numpy()
        assert rel_err(got, ref) <= F32_TOL


@pytest.mark.parametrize("dtype,scheme,rec", [(torch.float32, "explicit", "plain"),
                                              (torch.float32, "implicit", "plain"),
                                              (torch.float32, "explicit", "band"),
                                              (torch.float32, "implicit", "band"),
                                              (torch.float64, "explicit", "plain")])
def test_rbf_backward_matches_oracle(dtype, scheme, rec):
    """The RBF lift's gradient: the adjoint sweep (one block per pair, or the
    band form's chained reverse sweep), then the chain rule through the second
    difference of kappa over the points."""
    sigk = S()
    rec = sigk.REC_PLAIN if rec == "plain" else sigk.REC_BAND
    lam, d, L, M, sigma = 1, 7, 50, 40, 0.8
    Bx, By = 4, 3
    X32, X64 = inputs.f32(inputs.random_paths(6700, Bx, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(6701, By, M, d, time_channel=True))
    gout = np.random.default_rng(67).normal(size=(Bx, By))
    kw = dict(scheme=scheme, static_kernel="rbf", sigma=sigma)
    rX, rY = oracle.gram_grad(X64, Y64, lam, gout, **kw)
    Xd = to_dev(X32 if dtype == torch.float32 else X64, dtype)
    Yd = to_dev(Y32 if dtype == torch.float32 else Y64, dtype)
    v = rbf(sigma, scheme)
    dX, dY = sigk.gram_backward(to_dev(gout, dtype), Xd, Yd, lam, variant=v, rec=rec)
    tol = GRAD_TOL if dtype == torch.float32 else 1e-10
    assert grad_err(dX.cpu(), rX) <= tol
    assert grad_err(dY.cpu(), rY) <= tol
    g = np.random.default_rng(68).normal(size=3)
    pX, pY = oracle.pairs_grad(X64[:3], Y64, lam, g, **kw)
    dXp, dYp = sigk.pairs_backward(to_dev(g, dtype), Xd[:3], Yd, lam, variant=v, rec=rec)
    assert grad_err(dXp.cpu(), pX) <= tol
    assert grad_err(dYp.cpu(), pY) <= tol


def test_rbf_autograd_and_mmd():
    sigk = S()
    lam, d, L, B, sigma = 1, 5, 40, 4, 1.1
    X32, X64 = inputs.f32(inputs.random_paths(6800, B, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(6801, B, L, d, time_channel=True))
    v = rbf(sigma)
    X = to_dev(X32).requires_grad_(True)
    loss = sigk.mmd2_loss(X, to_dev(Y32), lam, variant=v)
    kw = dict(static_kernel="rbf", sigma=sigma)
    m = B
    Kxx = oracle.gram(X64, X64, lam, **kw)
    Kyy = oracle.gram(Y64, Y64, lam, **kw)
    Kxy = oracle.gram(X64, Y64, lam, **kw)
    want = ((Kxx.sum() - np.trace(Kxx)) / (m * (m - 1)) + (Kyy.sum() - np.trace(Kyy)) / (m * (m - 1))
            - 2 * Kxy.sum() / (m * m))
    assert abs(float(loss.detach()) - want) <= 1e-5 * max(1.0, abs(want))
    loss.backward()
    gxx = np.full((m, m), 1.0 / (m * (m - 1)))
    np.fill_diagonal(gxx, 0.0)
    a, b = oracle.gram_grad(X64, X64, lam, gxx, **kw)
    c, _ = oracle.gram_grad(X64, Y64, lam, np.full((m, m), -2.0 / (m * m)), want_dy=False, **kw)
    assert grad_err(X.grad.cpu(), a + b + c) <= GRAD_TOL


def test_rbf_unsupported_combinations():
    sigk = S()
    X = to_dev(inputs.random_paths(6900, 3, 30, 4, time_channel=True))
    v = rbf(1.0)
    with pytest.raises(sigk.SigkError) as ei:   # no tensor-core path for the lift
        sigk.gram(X, X, 1, schedule=sigk.Schedule(sigk.REC_STRIP, 0, sigk.COEF_TC), variant=v)
    assert ei.value.status == sigk.SIGK_EUNSUPPORTED
    with pytest.raises(sigk.SigkError) as ei:   # no strip backward for the lift
        sigk.gram_backward(torch.ones(3, 3, device="cuda"), X, X, 1, rec=sigk.REC_STRIP, variant=v)
    assert ei.value.status == sigk.SIGK_EUNSUPPORTED
    Xl = to_dev(inputs.random_paths(6901, 3, 600, 4, time_channel=True))
    with pytest.raises(sigk.SigkError) as ei:   # the symmetric backward needs the band form
        sigk.gram_backward(torch.ones(3, 3, device="cuda"), Xl, Xl, 1, symmetric=True, variant=v)
    assert ei.value.status == sigk.SIGK_EUNSUPPORTED


@pytest.mark.parametrize("lam,L,d,sigma", [(1, 60, 6, 0.9), (0, 130, 33, 1.7), (2, 33, 3, 0.6)])
def test_rbf_symmetric_gram_backward_in_the_band_form(lam, L, d, sigma):
    """The symmetric Gram's backward with the lift (pairs i <= j, the
    derivative through both arguments), against the oracle's gradient of the
    full Gram through both arguments; and autograd through the symmetric
    forward."""
    sigk = S()
    B = 6
    X32, X64 = inputs.f32(inputs.random_paths(6950 + L, B, L, d, time_channel=True))
    gout = np.random.default_rng(6951).normal(size=(B, B))
    kw = dict(static_kernel="rbf", sigma=sigma)
    rX, rY = oracle.gram_grad(X64, X64, lam, gout, **kw)
    v = rbf(sigma)
    dX, none = sigk.gram_backward(to_dev(gout), to_dev(X32), to_dev(X32), lam, symmetric=True, variant=v)
    assert none is None
    assert grad_err(dX.cpu(), rX + rY) <= GRAD_TOL
    X = to_dev(X32).requires_grad_(True)
    K = sigk.SigKernelGram.apply(X, X, lam, v)
    K.backward(to_dev(gout))
    assert grad_err(X.grad.cpu(), rX + rY) <= GRAD_TOL


def test_rbf_mmd_loss_in_the_band_form():
    """The lifted MMD^2 loss of 8 vs 8 paths (L = 96, d = 12, drift), whose
    fused value-and-gradient calls run the band backward: value and dL/dX
    against the oracle."""
    sigk = S()
    lam, sigma = 1, 1.3
    w = inputs.mmd_batches(B=8, L=96, d=12)
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    v = rbf(sigma)
    X = to_dev(X32).requires_grad_(True)
    loss = sigk.mmd2_loss(X, to_dev(Y32), lam, variant=v)
    kw = dict(static_kernel="rbf", sigma=sigma)
    m = 8
    Kxx = oracle.gram(X64, X64, lam, **kw)
    Kyy = oracle.gram(Y64, Y64, lam, **kw)
    Kxy = oracle.gram(X64, Y64, lam, **kw)
    want = ((Kxx.sum() - np.trace(Kxx)) / (m * (m - 1)) + (Kyy.sum() - np.trace(Kyy)) / (m * (m - 1))
            - 2 * Kxy.sum() / (m * m))
    assert abs(float(loss.detach()) - want) <= 1e-5 * max(1.0, abs(want))
    loss.backward()
    gxx = np.full((m, m), 1.0 / (m * (m - 1)))
    np.fill_diagonal(gxx, 0.0)
    a, b = oracle.gram_grad(X64, X64, lam, gxx, **kw)
    c, _ = oracle.gram_grad(X64, Y64, lam, np.full((m, m), -2.0 / (m * m)), want_dy=False, **kw)
    assert grad_err(X.grad.cpu(), a + b + c) <= GRAD_TOL
