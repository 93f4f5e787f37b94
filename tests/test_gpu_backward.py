"""Parity of the CUDA adjoint (reverse-mode derivative of the discrete scheme)
with the FP64 oracle's own gradient, and against central finite differences;
the MMD^2 estimator and its gradient.  Bars: FP64 <= 1e-10 relative to the
largest gradient entry, FP32 <= 1e-4 (the gradient tolerance the workload
states), FD <= 1e-4 relative."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    from paper_2006_14794_gb300 import sigk
    sigk.lib()


def S():
    from paper_2006_14794_gb300 import sigk
    return sigk


def grad_err(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30))


@pytest.mark.parametrize("lam,L,M,d", [(0, 9, 12, 3), (1, 32, 32, 3), (2, 17, 11, 4), (1, 40, 25, 8)])
def test_pairs_backward_matches_oracle(lam, L, M, d):
    B = 7
    X32, X64 = inputs.f32(inputs.random_paths(500 + lam, B, L, d, scale=2.0, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(600 + lam, B, M, d, scale=2.0, time_channel=True))
    g = np.random.default_rng(1).normal(size=B)
    rX, rY = oracle.pairs_grad(X64, Y64, lam, g)
    dX, dY = S().pairs_backward(to_dev(g, torch.float64), to_dev(X64, torch.float64),
                                to_dev(Y64, torch.float64), lam)
    assert grad_err(dX.cpu(), rX) <= 1e-10
    assert grad_err(dY.cpu(), rY) <= 1e-10
    dX, dY = S().pairs_backward(to_dev(g), to_dev(X32), to_dev(Y32), lam)
    assert grad_err(dX.cpu(), rX) <= 1e-4
    assert grad_err(dY.cpu(), rY) <= 1e-4


def test_gram_backward_matches_oracle():
    w = inputs.gram_small()
    lam = w["dyadic_order"]
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    gout = np.random.default_rng(2).normal(size=(8, 8))
    rX, rY = oracle.gram_grad(X64, Y64, lam, gout)
    dX, dY = S().gram_backward(to_dev(gout, torch.float64), to_dev(X64, torch.float64),
                               to_dev(Y64, torch.float64), lam)
    assert grad_err(dX.cpu(), rX) <= 1e-10
    assert grad_err(dY.cpu(), rY) <= 1e-10
    dX, dY = S().gram_backward(to_dev(gout), to_dev(X32), to_dev(Y32), lam)
    assert grad_err(dX.cpu(), rX) <= 1e-4
    assert grad_err(dY.cpu(), rY) <= 1e-4


def test_backward_uneven_lengths_swap_sides():
    # L > M: the kernel puts the shorter path on the rows; gradients must land on
    # the right tensors
    X32, X64 = inputs.f32(inputs.random_paths(700, 3, 30, 3, scale=2.0))
    Y32, Y64 = inputs.f32(inputs.random_paths(701, 4, 9, 3, scale=2.0))
    gout = np.random.default_rng(3).normal(size=(3, 4))
    rX, rY = oracle.gram_grad(X64, Y64, 1, gout)
    dX, dY = S().gram_backward(to_dev(gout, torch.float64), to_dev(X64, torch.float64),
                               to_dev(Y64, torch.float64), 1)
    assert grad_err(dX.cpu(), rX) <= 1e-10
    assert grad_err(dY.cpu(), rY) <= 1e-10


def test_autograd_against_central_differences():
    # FP64 autograd through the library vs central differences (h = 1e-6) of the
    # library's own FP64 forward, on 24 seeded coordinates
    X = to_dev(inputs.random_paths(710, 3, 12, 3, scale=2.0), torch.float64).requires_grad_(True)
    Y = to_dev(inputs.random_paths(711, 2, 10, 3, scale=2.0), torch.float64)
    W = to_dev(np.random.default_rng(4).normal(size=(3, 2)), torch.float64)
    loss = (S().SigKernelGram.apply(X, Y, 1) * W).sum()
    loss.backward()
    g = X.grad.cpu().numpy()
    rng = np.random.default_rng(5)
    h = 1e-6
    with torch.no_grad():
        for _ in range(24):
            idx = tuple(int(rng.integers(0, s)) for s in X.shape)
            Xp, Xm = X.detach().clone(), X.detach().clone()
            Xp[idx] += h
            Xm[idx] -= h
            fd = ((S().gram(Xp, Y, 1) * W).sum() - (S().gram(Xm, Y, 1) * W).sum()).item() / (2 * h)
            assert abs(g[idx] - fd) <= 1e-4 * max(abs(fd), np.abs(g).max() * 1e-2)


def test_mmd2_matches_oracle_and_its_gradient():
    X64 = inputs.random_paths(720, 6, 14, 3, scale=2.0)
    Y64 = inputs.random_paths(721, 5, 14, 3, scale=2.0) + 0.3 * np.linspace(0, 1, 14)[None, :, None]
    lam = 1
    ref = oracle.mmd2(X64, Y64, lam)
    rg = oracle.mmd2_grad_x(X64, Y64, lam)
    X = to_dev(X64, torch.float64).requires_grad_(True)
    Y = to_dev(Y64, torch.float64)
    val = S().mmd2_loss(X, Y, lam)
    assert abs(val.item() - ref) <= 1e-11 * max(1.0, abs(ref))
    val.backward()
    assert grad_err(X.grad.cpu(), rg) <= 1e-10
    # FP32
    X32 = to_dev(X64).requires_grad_(True)
    v32 = S().mmd2_loss(X32, to_dev(Y64), lam)
    v32.backward()
    assert abs(v32.item() - ref) <= 1e-5
    assert grad_err(X32.grad.cpu(), rg) <= 1e-4


def test_mmd_workload_gradient_sampled():
    # the MMD^2 workload (128 vs 128 paths, L=256, d=32, drift 0.1, dyadic
    # order 1) at reduced batch (8 vs 8), gradient checked against the oracle
    w = inputs.mmd_batches(B=8)
    lam = w["dyadic_order"]
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    X = to_dev(X32).requires_grad_(True)
    v = S().mmd2_loss(X, to_dev(Y32), lam)
    v.backward()
    ref = oracle.mmd2(X64, Y64, lam)
    assert abs(v.item() - ref) <= 1e-5 * max(1.0, abs(ref))
    rg = oracle.mmd2_grad_x(X64, Y64, lam)
    assert grad_err(X.grad.cpu(), rg) <= 1e-4


def test_workspace_too_small_is_an_error():
    import ctypes
    lib = S().lib()
    X = to_dev(inputs.random_paths(730, 2, 10, 3))
    g = torch.ones(2, device="cuda")
    dX = torch.empty_like(X)
    o = S().SigkOpts()
    need = lib.sigk_workspace_bytes(S().OP_PAIRS_BACKWARD, 2, 0, 10, 10, 3, 1, 0, ctypes.byref(o))
    assert need > 0
    ws = torch.empty(need - 1, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    r = lib.sigk_pairs_backward(g.data_ptr(), X.data_ptr(), X.data_ptr(), 2, 10, 10, 3, 1, 0,
                                ctypes.byref(o), dX.data_ptr(), None, ws.data_ptr(), need - 1, st)
    assert r == S().SIGK_ENOMEM_WS


@pytest.mark.parametrize("lam,L,M,d", [(0, 700, 300, 3), (1, 40, 25, 8), (2, 150, 160, 4), (3, 33, 70, 5)])
def test_strip_backward_matches_oracle(lam, L, M, d):
    # the strip path's adjoint (f32 by default, f64 on request), multi-strip
    # pairs included, against the oracle's gradient and the plain backward
    B = 3
    X32, X64 = inputs.f32(inputs.random_paths(800 + lam, B, L, d, scale=2.0, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(900 + lam, B, M, d, scale=2.0, time_channel=True))
    g = np.random.default_rng(6).normal(size=B)
    rX, rY = oracle.pairs_grad(X64, Y64, lam, g)
    dX, dY = S().pairs_backward(to_dev(g), to_dev(X32), to_dev(Y32), lam, rec=S().REC_STRIP)
    assert grad_err(dX.cpu(), rX) <= 1e-4
    assert grad_err(dY.cpu(), rY) <= 1e-4
    dX, dY = S().pairs_backward(to_dev(g, torch.float64), to_dev(X64, torch.float64),
                                to_dev(Y64, torch.float64), lam, rec=S().REC_CHAIN)
    assert grad_err(dX.cpu(), rX) <= 1e-10
    assert grad_err(dY.cpu(), rY) <= 1e-10
    pX, pY = S().pairs_backward(to_dev(g), to_dev(X32), to_dev(Y32), lam, rec=S().REC_PLAIN)
    assert grad_err(pX.cpu(), rX) <= 1e-4


def test_strip_backward_long_pair_at_dyadic_order_1():
    """One pair of the long-pair workload (L = M = 4096, d = 64, dyadic order
    1: 8190 x 8190 refined cells, 16 strips of 512 rows): the strip adjoint
    runs the forward backwards between checkpoints (every 64 steps in FP32,
    128 in FP64) instead of reading stored per-cell sums."""
    w = inputs.long_pairs(B=1)
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    g = np.array([0.75])
    rX, rY = oracle.pairs_grad(X64, Y64, 1, g)
    dX, dY = S().pairs_backward(to_dev(g), to_dev(X32), to_dev(Y32), 1, rec=S().REC_STRIP, check_status=True)
    assert grad_err(dX.cpu(), rX) <= 1e-4
    assert grad_err(dY.cpu(), rY) <= 1e-4
    dX, dY = S().pairs_backward(to_dev(g, torch.float64), to_dev(X64, torch.float64),
                                to_dev(Y64, torch.float64), 1, rec=S().REC_CHAIN, check_status=True)
    assert grad_err(dX.cpu(), rX) <= 1e-10
    assert grad_err(dY.cpu(), rY) <= 1e-10
