"""Backward calls that add into the caller's gradient buffers
(sigk_opts.accumulate) on every backward path, and the scalar chain rule
(sigk_scale_grad) that the MMD^2 loss applies to its stored gradients.

A loss that sums several Grams of the same paths (the unbiased MMD^2 adds
Kxx's and Kxy's gradients into dX) needs the second call to add to the first
call's result, and the loss's upstream derivative to scale the sum.  Both
happen in the library, so the binding does no arithmetic."""
import numpy as np
import pytest
import torch

from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu


def S():
    from paper_2006_14794_gb300 import sigk
    return sigk


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    S().lib()


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


# (label, Bx, By, L, M, d, lambda, dtype, rec, symmetric): the band form
# (plain Gram and symmetric Gram), the strip path and the plain backward
CASES = [
    ("band", 6, 5, 40, 40, 8, 1, torch.float32, 0, False),
    ("band-sym", 7, 7, 33, 33, 6, 1, torch.float32, 0, True),
    ("strip", 4, 3, 50, 70, 8, 1, torch.float32, 3, False),
    ("plain-f64", 4, 5, 30, 26, 3, 2, torch.float64, 0, False),
    ("strip-f64", 3, 4, 44, 31, 5, 1, torch.float64, 1, False),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gram_backward_accumulates(case):
    _, Bx, By, L, M, d, lam, dt, rec, sym = case
    X = to_dev(inputs.random_paths(1200, Bx, L, d, scale=2.0, time_channel=True), dt)
    Y = X if sym else to_dev(inputs.random_paths(1201, By, M, d, scale=2.0, time_channel=True), dt)
    g = to_dev(np.random.default_rng(1202).normal(size=(Bx, By)), dt)
    fX, fY = S().gram_backward(g, X, Y, lam, rec=rec, symmetric=sym)
    P = torch.randn_like(X)
    Q = None if sym else torch.randn_like(Y)
    aX, aY = S().gram_backward(g, X, Y, lam, rec=rec, symmetric=sym, dX=P.clone(),
                               dY=None if sym else Q.clone(), accumulate=True)
    tol = 1e-6 if dt == torch.float32 else 1e-13
    assert _rel(aX, P + fX) <= tol
    if not sym:
        assert _rel(aY, Q + fY) <= tol


def test_pairs_backward_accumulates():
    for dt, rec in ((torch.float32, 0), (torch.float64, 0), (torch.float32, 3)):
        X = to_dev(inputs.random_paths(1210, 9, 37, 4, scale=2.0, time_channel=True), dt)
        Y = to_dev(inputs.random_paths(1211, 9, 29, 4, scale=2.0, time_channel=True), dt)
        g = to_dev(np.random.default_rng(1212).normal(size=9), dt)
        fX, fY = S().pairs_backward(g, X, Y, 1, rec=rec)
        P, Q = torch.randn_like(X), torch.randn_like(Y)
        aX, aY = S().pairs_backward(g, X, Y, 1, rec=rec, dX=P.clone(), dY=Q.clone(), accumulate=True)
        tol = 1e-6 if dt == torch.float32 else 1e-13
        assert _rel(aX, P + fX) <= tol, (dt, rec)
        assert _rel(aY, Q + fY) <= tol, (dt, rec)


def test_value_and_grad_accumulates_and_keeps_the_values():
    X = to_dev(inputs.random_paths(1220, 6, 48, 8, scale=2.0, time_channel=True))
    Y = to_dev(inputs.random_paths(1221, 5, 48, 8, scale=2.0, time_channel=True))
    g = to_dev(np.random.default_rng(1222).normal(size=(6, 5)))
    K0, fX, fY = S().gram_value_and_grad(g, X, Y, 1)
    P, Q = torch.randn_like(X), torch.randn_like(Y)
    K1, aX, aY = S().gram_value_and_grad(g, X, Y, 1, dX=P.clone(), dY=Q.clone(), accumulate=True)
    assert torch.equal(K0, K1)
    assert torch.equal(aX, P + fX)
    assert torch.equal(aY, Q + fY)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_scale_grad(dt):
    x = torch.randn(1000003, dtype=dt, device="cuda")
    s = torch.tensor([-2.75], dtype=dt, device="cuda")
    assert torch.equal(S().scale_grad(s, x), s * x)


def test_mmd2_loss_gradient_scales_with_the_upstream_derivative():
    w = inputs.mmd_batches(B=12, L=40, d=6)
    X32, _ = inputs.f32(w["X"])
    Y32, _ = inputs.f32(w["Y"])
    Yd = to_dev(Y32).requires_grad_(True)
    grads = []
    for up in (1.0, -3.5):
        X = to_dev(X32).requires_grad_(True)
        Yd.grad = None
        v = S().mmd2_loss(X, Yd, 1)
        (up * v).backward()
        grads.append((X.grad.clone(), Yd.grad.clone()))
    assert _rel(grads[1][0], -3.5 * grads[0][0]) <= 1e-6
    assert _rel(grads[1][1], -3.5 * grads[0][1]) <= 1e-6
