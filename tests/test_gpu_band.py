"""The band form (coefficients formed by a contraction kernel into a banded
buffer, read by the register chain): parity with the FP64 oracle through the C
ABI, across every (rows per lane, dyadic order) instance, pair turnovers within
a warp's chain, virtual rows and columns, both orientations, symmetric Grams,
and the shapes of the 128 x 128 MMD workload."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    from paper_2006_14794_gb300 import sigk
    sigk.lib()


def S():
    from paper_2006_14794_gb300 import sigk
    return sigk


def band(R):
    return S().Schedule(S().REC_BAND, R, 0)


@pytest.mark.parametrize("R,lam,L,M,d", [
    (16, 1, 256, 256, 32),   # the MMD shape: 510 refined rows, 8 coarse rows per lane
    (16, 1, 200, 300, 24),   # virtual rows (398 of 512) and virtual columns
    (16, 2, 100, 77, 5),     # 4 coarse rows per lane
    (16, 3, 60, 61, 3),      # 2 coarse rows per lane
    (8, 0, 230, 256, 40),    # dyadic order 0, 8 coarse rows per lane
    (8, 1, 129, 140, 17),
    (8, 2, 40, 33, 9),
    (4, 0, 100, 120, 64),
    (4, 1, 60, 90, 33),
])
def test_band_gram_matches_oracle(R, lam, L, M, d):
    # enough pairs that warps chain several of them (pair turnovers inside a warp)
    Bx, By = 7, 9
    X32, X64 = inputs.f32(inputs.random_paths(3100 + R + lam, Bx, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(3200 + R + lam, By, M, d, time_channel=True))
    ref = oracle.gram(X64, Y64, lam)
    got = S().gram(to_dev(X32), to_dev(Y32), lam, schedule=band(R)).cpu().numpy()
    assert rel_err(got, ref) <= F32_TOL
    # the other orientation (rows refine the shorter path either way)
    got_t = S().gram(to_dev(Y32), to_dev(X32), lam, schedule=band(R)).cpu().numpy()
    assert rel_err(got_t, ref.T) <= F32_TOL


def test_band_pairs_both_orders_and_long_chains():
    lam, d = 1, 32
    B = 3000   # ~2-3 pairs per warp at 12 warps per SM
    X32, X64 = inputs.f32(inputs.random_paths(3300, B, 40, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(3301, B, 35, d, time_channel=True))
    ref = oracle.pairs(X64, Y64, lam)
    got = S().pairs(to_dev(X32), to_dev(Y32), lam, schedule=band(16)).cpu().numpy()
    assert rel_err(got, ref) <= F32_TOL
    got2 = S().pairs(to_dev(Y32), to_dev(X32), lam, schedule=band(16)).cpu().numpy()
    assert rel_err(got2, ref) <= F32_TOL


def test_band_symmetric_gram():
    lam, d = 1, 32
    X32, X64 = inputs.f32(inputs.random_paths(3400, 11, 129, d, time_channel=True))
    ref = oracle.gram(X64, X64, lam)
    got = S().gram(to_dev(X32), to_dev(X32), lam, symmetric=True, schedule=band(8)).cpu().numpy()
    assert rel_err(got, ref) <= F32_TOL
    assert np.array_equal(got, got.T)


def test_band_is_the_default_for_wide_short_pairs():
    """d = 32 has no inline-product chain instance: AUTO takes the band form,
    which needs workspace; its result equals the forced schedule's bit for bit."""
    sigk = S()
    lam, d = 1, 32
    w = inputs.mmd_batches(B=6)
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    auto = sigk.gram(to_dev(X32), to_dev(Y32), lam).cpu().numpy()
    forced = sigk.gram(to_dev(X32), to_dev(Y32), lam, schedule=band(16)).cpu().numpy()
    assert np.array_equal(auto, forced)
    assert rel_err(auto, oracle.gram(X64, Y64, lam)) <= F32_TOL


def test_band_refuses_what_it_cannot_do():
    sigk = S()
    X = to_dev(inputs.random_paths(3500, 2, 600, 4, time_channel=True))
    with pytest.raises(sigk.SigkError) as ei:   # 599 rows do not fit a warp
        sigk.pairs(X, X, 0, schedule=band(16))
    assert ei.value.status == sigk.SIGK_EUNSUPPORTED
    X64 = to_dev(inputs.random_paths(3501, 2, 60, 4, time_channel=True), torch.float64)
    with pytest.raises(sigk.SigkError) as ei:
        sigk.pairs(X64, X64, 1, schedule=band(16))
    assert ei.value.status == sigk.SIGK_EUNSUPPORTED


# ------------------------------------------------------------------ backward

def grad_err(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30))


GRAD_TOL = 1e-4


@pytest.mark.parametrize("R,lam,L,M,d", [
    (16, 1, 256, 256, 32),   # the MMD shape
    (16, 1, 120, 200, 24),   # virtual rows and columns
    (16, 2, 70, 77, 5),
    (16, 3, 40, 41, 3),
    (8, 0, 230, 256, 40),
    (8, 1, 100, 90, 17),     # rows refine the second path
    (8, 2, 40, 33, 9),
    (4, 0, 100, 120, 6),
    (4, 1, 60, 70, 33),
])
def test_band_gram_backward_matches_oracle(R, lam, L, M, d):
    """The reversible adjoint (forward state undone in place between
    checkpoints) against the oracle's exact gradient, with pair turnovers
    inside each warp's chain."""
    Bx, By = 5, 6
    X32, X64 = inputs.f32(inputs.random_paths(3600 + R + lam, Bx, L, d, scale=2.0, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(3700 + R + lam, By, M, d, scale=2.0, time_channel=True))
    gout = np.random.default_rng(37).normal(size=(Bx, By))
    rX, rY = oracle.gram_grad(X64, Y64, lam, gout)
    s = S().Schedule(S().REC_BAND, R, 0)
    dX, dY = S().gram_backward(to_dev(gout), to_dev(X32), to_dev(Y32), lam, schedule=s)
    assert grad_err(dX.cpu(), rX) <= GRAD_TOL
    assert grad_err(dY.cpu(), rY) <= GRAD_TOL
    # only one side requested
    dX1, none = S().gram_backward(to_dev(gout), to_dev(X32), to_dev(Y32), lam, need_dy=False, schedule=s)
    assert none is None and torch.equal(dX1, dX)


@pytest.mark.parametrize("L,M", [(60, 60), (80, 50), (33, 90)])
def test_band_pairs_backward_matches_oracle(L, M):
    lam, d, B = 1, 20, 700   # several pairs per warp
    X32, X64 = inputs.f32(inputs.random_paths(3800 + L, B, L, d, scale=2.0, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(3900 + M, B, M, d, scale=2.0, time_channel=True))
    g = np.random.default_rng(39).normal(size=B)
    rX, rY = oracle.pairs_grad(X64, Y64, lam, g)
    dX, dY = S().pairs_backward(to_dev(g), to_dev(X32), to_dev(Y32), lam, schedule=band(16))
    assert grad_err(dX.cpu(), rX) <= GRAD_TOL
    assert grad_err(dY.cpu(), rY) <= GRAD_TOL


def test_band_backward_is_the_default_and_agrees_with_the_strip_adjoint():
    sigk = S()
    w = inputs.mmd_batches(B=5)
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    gout = np.random.default_rng(40).normal(size=(5, 5))
    auto = sigk.gram_backward(to_dev(gout), to_dev(X32), to_dev(Y32), 1)
    band_ = sigk.gram_backward(to_dev(gout), to_dev(X32), to_dev(Y32), 1, schedule=band(16))
    strip = sigk.gram_backward(to_dev(gout), to_dev(X32), to_dev(Y32), 1, rec=sigk.REC_STRIP)
    for a_, b_, s_ in zip(auto, band_, strip):
        assert torch.equal(a_, b_)
        assert grad_err(a_.cpu(), s_.cpu()) <= GRAD_TOL
    rX, rY = oracle.gram_grad(X64, Y64, 1, gout)
    assert grad_err(auto[0].cpu(), rX) <= GRAD_TOL
    assert grad_err(auto[1].cpu(), rY) <= GRAD_TOL


@pytest.mark.parametrize("lam,L,d", [(1, 256, 32), (1, 100, 9), (2, 60, 5)])
def test_band_symmetric_backward_matches_oracle(lam, L, d):
    """Pairs i <= j only: the derivative through both arguments of a Gram of X
    with itself, for a non-symmetric incoming gradient."""
    sigk = S()
    B = 7
    X32, X64 = inputs.f32(inputs.random_paths(4100 + L, B, L, d, scale=2.0, time_channel=True))
    gout = np.random.default_rng(41).normal(size=(B, B))
    rX, rY = oracle.gram_grad(X64, X64, lam, gout)
    dX, none = sigk.gram_backward(to_dev(gout), to_dev(X32), to_dev(X32), lam, symmetric=True)
    assert none is None
    assert grad_err(dX.cpu(), rX + rY) <= GRAD_TOL
    # the symmetric forward and autograd through it
    X = to_dev(X32).requires_grad_(True)
    K = sigk.SigKernelGram.apply(X, X, lam)
    assert rel_err(K.detach().cpu().numpy(), oracle.gram(X64, X64, lam)) <= F32_TOL
    K.backward(to_dev(gout))
    assert grad_err(X.grad.cpu(), rX + rY) <= GRAD_TOL


@pytest.mark.parametrize("R,lam,L,M,d,sym", [
    (16, 1, 256, 256, 32, False),   # the MMD workload's shape
    (16, 1, 256, 256, 32, True),
    (8, 1, 100, 90, 17, False),     # rows refine the second path
    (8, 2, 40, 40, 9, True),
    (4, 0, 60, 70, 6, False),       # d <= 16: sigk_gram's default is the chain kernel
])
def test_gram_value_and_grad_equals_the_two_calls(R, lam, L, M, d, sym):
    """sigk_gram_value_and_grad: the backward's forward sweep writes the
    values; gradients identical to sigk_gram_backward's, values identical to
    sigk_gram's on the same schedule and within the FP32 bar of the oracle
    (sigk_gram's default for d <= 16, the chain kernel, rounds differently)."""
    sigk = S()
    Bx, By = 7, (7 if sym else 6)
    X32, X64 = inputs.f32(inputs.random_paths(5100 + R + lam, Bx, L, d, scale=2.0, time_channel=True))
    Y32, Y64 = (X32, X64) if sym else inputs.f32(
        inputs.random_paths(5200 + R + lam, By, M, d, scale=2.0, time_channel=True))
    gout = to_dev(np.random.default_rng(51).normal(size=(Bx, By)))
    X, Y = to_dev(X32), to_dev(Y32)
    s = sigk.Schedule(sigk.REC_BAND, R, 0)
    K, dX, dY = sigk.gram_value_and_grad(gout, X, Y, lam, schedule=s, symmetric=sym)
    rX, rY = sigk.gram_backward(gout, X, Y, lam, schedule=s, symmetric=sym)
    assert torch.equal(dX, rX)
    assert (dY is None and rY is None) if sym else torch.equal(dY, rY)
    assert torch.equal(K, sigk.gram(X, Y, lam, symmetric=sym, schedule=s))
    assert rel_err(K.cpu().numpy(), oracle.gram(X64, Y64, lam)) <= F32_TOL


def test_mmd2_loss_fused_equals_composed():
    """mmd2_loss with a gradient wanted takes the fused path; the composition
    of the Grams' autograd functions gives the same loss and gradients."""
    sigk = S()
    w = inputs.mmd_batches(B=12, L=64)
    lam = w["dyadic_order"]
    X = to_dev(inputs.f32(w["X"])[0]).requires_grad_(True)
    Y = to_dev(inputs.f32(w["Y"])[0]).requires_grad_(True)
    v = sigk.mmd2_loss(X, Y, lam)
    def fn_name(t):   # the node under the [0] select
        return type(t.grad_fn.next_functions[0][0]).__name__

    assert "MMD2Fused" in fn_name(v)
    (3.0 * v).backward()
    X2 = X.detach().clone().requires_grad_(True)
    Y2 = Y.detach().clone().requires_grad_(True)
    Kxx = sigk.SigKernelGram.apply(X2, X2, lam, None)
    Kyy = sigk.SigKernelGram.apply(Y2, Y2, lam, None)
    Kxy = sigk.SigKernelGram.apply(X2, Y2, lam, None)
    v2 = sigk._MMD2.apply(Kxx, Kyy, Kxy)[0]
    (3.0 * v2).backward()
    assert abs(v.item() - v2.item()) <= 1e-6 * max(1.0, abs(v2.item()))
    # the fused path contracts dk/dc for unit weights and scales the result by
    # the upstream 3 afterwards; the composed one contracts the scaled dk/dc.
    # The chain-rule contraction's split-TF32 products keep about 22 bits of
    # each operand, so the two orders agree to a few units of 1e-7, not bit
    # for bit
    assert grad_err(X.grad.cpu(), X2.grad.cpu()) <= 1e-5
    assert grad_err(Y.grad.cpu(), Y2.grad.cpu()) <= 1e-5
    # outside the band form (FP64) the composition runs
    X64 = X.detach().double().requires_grad_(True)
    v64 = sigk.mmd2_loss(X64, Y.detach().double(), lam)
    assert "MMD2Fused" not in fn_name(v64)
    (3.0 * v64).backward()
    assert grad_err(X64.grad.cpu(), X2.grad.cpu()) <= 1e-4


def test_symmetric_backward_argument_checks():
    sigk = S()
    X = to_dev(inputs.random_paths(4200, 3, 20, 3))
    Y = to_dev(inputs.random_paths(4201, 4, 20, 3))
    with pytest.raises(sigk.SigkError) as ei:   # different batches
        sigk.gram_backward(torch.ones(3, 4, device="cuda"), X, Y, 1, symmetric=True)
    assert ei.value.status == sigk.SIGK_EINVAL


@pytest.mark.parametrize("R,lam,L,M,d", [
    (16, 1, 256, 256, 32),   # 8 coarse rows per lane: two 128-row tiles
    (8, 0, 230, 256, 40),    # 8 per lane, d not a multiple of 8
    (4, 0, 100, 120, 64),    # 4 per lane: one tile
    (4, 1, 60, 90, 33),      # 2 per lane: half a tile
])
def test_band_tcgen05_coefficients_match_oracle(R, lam, L, M, d):
    """The band's coefficients from split-TF32 tcgen05 MMAs (coef_path 3),
    forward and backward, against the oracle."""
    sigk = S()
    Bx, By = 5, 6
    X32, X64 = inputs.f32(inputs.random_paths(4800 + R + lam, Bx, L, d, scale=2.0, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(4900 + R + lam, By, M, d, scale=2.0, time_channel=True))
    s = sigk.Schedule(sigk.REC_BAND, R, sigk.COEF_TC5)
    got = sigk.gram(to_dev(X32), to_dev(Y32), lam, schedule=s, check_status=True).cpu().numpy()
    assert rel_err(got, oracle.gram(X64, Y64, lam)) <= F32_TOL
    gout = np.random.default_rng(48).normal(size=(Bx, By))
    rX, rY = oracle.gram_grad(X64, Y64, lam, gout)
    dX, dY = sigk.gram_backward(to_dev(gout), to_dev(X32), to_dev(Y32), lam, schedule=s)
    assert grad_err(dX.cpu(), rX) <= GRAD_TOL
    assert grad_err(dY.cpu(), rY) <= GRAD_TOL


@pytest.mark.parametrize("L,M,d,sym", [
    (256, 256, 32, False),   # the MMD shape: 255-row blocks across 128-row tiles
    (100, 120, 64, False),   # N = 64: two TMEM read-backs
    (77, 77, 48, True),      # N = 48 (padded to 48 of 64 columns); triangle skipping
    (33, 41, 3, False),      # N = 3, padded to 16; K tails in every chunk
])
def test_chain_rule_tensor_cores_match_the_fma_contraction(L, M, d, sym):
    """The Gram backward's chain rule (d dx = Gbar dy, d dy = Gbar^T dx) as
    split-TF32 tcgen05 MMAs (coef_path 3) and on the FP32 pipe (coef_path 1),
    both against the oracle's gradient."""
    sigk = S()
    Bx, By = 9, (9 if sym else 7)
    X32, X64 = inputs.f32(inputs.random_paths(4300 + L, Bx, L, d, scale=2.0, time_channel=True))
    Y32, Y64 = (X32, X64) if sym else inputs.f32(inputs.random_paths(4400 + M, By, M, d, scale=2.0,
                                                                        time_channel=True))
    gout = np.random.default_rng(43).normal(size=(Bx, By))
    rX, rY = oracle.gram_grad(X64, Y64, 1, gout)
    if sym:
        rX, rY = rX + rY, None
    out = {}
    for name, cp in (("tc", sigk.COEF_TC5), ("fma", sigk.COEF_FMA)):
        s = sigk.Schedule(sigk.REC_BAND, 0, cp)
        out[name] = sigk.gram_backward(to_dev(gout), to_dev(X32), to_dev(Y32), 1, schedule=s, symmetric=sym)
    errs = {}
    for name in out:
        errs[name] = grad_err(out[name][0].cpu(), rX)
        assert errs[name] <= GRAD_TOL, name
        if not sym:
            assert grad_err(out[name][1].cpu(), rY) <= GRAD_TOL, name
    # split-TF32 keeps about 22 bits of each operand (FP32: 24), and a
    # gradient entry sums thousands of products of both signs: the two
    # contractions agree to a few 1e-5 of the gradient's largest entry
    errs["tc-fma"] = grad_err(out["tc"][0].cpu(), out["fma"][0].cpu())
    print("chain rule errors (dX vs oracle; tensor cores vs FMA):", errs)
    assert errs["tc-fma"] <= 5e-5
