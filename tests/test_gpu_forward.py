"""Parity of the CUDA forward sweep with the FP64 oracle, through the C ABI.

FP32 results are compared with the oracle run on the same FP32 inputs promoted
to FP64, so the error measured is the kernel's own arithmetic.  Bars: relative
error <= 1e-5 for the FP32 recurrence, <= 1e-11 for the FP64 one (relative to
max(|k|, 1e-3))."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
F64_TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    from paper_2006_14794_gb300 import sigk
    sigk.lib()


def S():
    from paper_2006_14794_gb300 import sigk
    return sigk


# ------------------------------------------------------------ the small Gram

def test_gram_small_fp64_plain_and_fp32_chain():
    w = inputs.gram_small()
    lam = w["dyadic_order"]
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    ref64 = oracle.gram(w["X"], w["Y"], lam)
    got64 = S().gram(to_dev(w["X"], torch.float64), to_dev(w["Y"], torch.float64), lam).cpu().numpy()
    assert rel_err(got64, ref64) <= F64_TOL
    ref32 = oracle.gram(X64, Y64, lam)
    got32 = S().gram(to_dev(X32), to_dev(Y32), lam).cpu().numpy()
    assert rel_err(got32, ref32) <= F32_TOL
    plain32 = S().gram(to_dev(X32), to_dev(Y32), lam, rec=S().REC_PLAIN).cpu().numpy()
    assert rel_err(plain32, ref32) <= F32_TOL


def test_straight_lines_small():
    w = inputs.gram_small()
    lam = w["dyadic_order"]
    ref = oracle.pairs(w["lines_x"], w["lines_y"], lam)
    got = S().pairs(to_dev(w["lines_x"], torch.float64), to_dev(w["lines_y"], torch.float64), lam)
    assert rel_err(got.cpu().numpy(), ref) <= F64_TOL
    x32, x64 = inputs.f32(w["lines_x"])
    y32, y64 = inputs.f32(w["lines_y"])
    got32 = S().pairs(to_dev(x32), to_dev(y32), lam).cpu().numpy()
    assert rel_err(got32, oracle.pairs(x64, y64, lam)) <= F32_TOL


# -------------------------------------------- chained kernel: shapes and tails

@pytest.mark.parametrize("lam,L,M,d", [
    (0, 33, 47, 3), (0, 100, 70, 2), (1, 20, 40, 4), (1, 129, 65, 8), (2, 17, 33, 8),
    (2, 128, 128, 8), (2, 60, 90, 5), (3, 9, 17, 16), (3, 33, 21, 4), (4, 5, 9, 8),
    (4, 17, 12, 3), (1, 200, 256, 16),
])
def test_pairs_fp32_matches_oracle(lam, L, M, d):
    B = 37   # ragged: not a multiple of any warp/pair chunk
    X32, X64 = inputs.f32(inputs.random_paths(100 + lam, B, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(200 + lam, B, M, d, time_channel=True))
    ref = oracle.pairs(X64, Y64, lam)
    got = S().pairs(to_dev(X32), to_dev(Y32), lam).cpu().numpy()
    assert rel_err(got, ref) <= F32_TOL


@pytest.mark.parametrize("Bx,By,L,M", [(5, 7, 40, 40), (9, 4, 65, 30), (3, 11, 20, 70)])
def test_gram_fp32_chain_and_plain(Bx, By, L, M):
    lam, d = 2, 8
    X32, X64 = inputs.f32(inputs.random_paths(300, Bx, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(301, By, M, d, time_channel=True))
    ref = oracle.gram(X64, Y64, lam)
    got = S().gram(to_dev(X32), to_dev(Y32), lam).cpu().numpy()
    assert got.shape == (Bx, By)
    assert rel_err(got, ref) <= F32_TOL
    plain = S().gram(to_dev(X32), to_dev(Y32), lam, rec=S().REC_PLAIN).cpu().numpy()
    assert rel_err(plain, ref) <= F32_TOL
    g64 = S().gram(to_dev(X64, torch.float64), to_dev(Y64, torch.float64), lam).cpu().numpy()
    assert rel_err(g64, ref) <= F64_TOL


def test_symmetric_gram():
    X32, X64 = inputs.f32(inputs.random_paths(310, 13, 50, 4, time_channel=True))
    ref = oracle.gram(X64, X64, 1)
    for rec in (S().REC_AUTO, S().REC_PLAIN):
        got = S().gram(to_dev(X32), to_dev(X32), 1, rec=rec, symmetric=True).cpu().numpy()
        assert rel_err(got, ref) <= F32_TOL
        assert np.array_equal(got, got.T)


def test_gram_256_sampled_entries():
    # the 256 x 256 Gram of 128-point, 8-channel paths at dyadic order 2 (the
    # benchmark's workload), in the benchmark's launch, checked on 200 sampled
    # entries against the oracle computed one by one
    w = inputs.gram_256()
    lam = w["dyadic_order"]
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    got = S().gram(to_dev(X32), to_dev(Y32), lam).cpu().numpy()
    rng = np.random.default_rng(7)
    idx = rng.integers(0, 256, size=(200, 2))
    idx = np.vstack([idx, [[0, 0], [255, 255], [0, 255], [255, 0]]])
    ref = np.array([oracle.sigkernel(X64[i], Y64[j], lam) for i, j in idx])
    assert rel_err(got[idx[:, 0], idx[:, 1]], ref) <= F32_TOL
    assert np.isfinite(got).all()


# ------------------------------------------------------------------ edge cases

def test_single_point_paths_give_one():
    X = to_dev(np.random.default_rng(0).normal(size=(4, 1, 3)))
    Y = to_dev(np.random.default_rng(1).normal(size=(4, 9, 3)))
    for lam in (0, 3):
        assert torch.all(S().pairs(X, Y, lam) == 1)
        assert torch.all(S().pairs(Y, X, lam) == 1)
        assert torch.all(S().gram(X, Y, lam) == 1)


def test_empty_batch():
    X = torch.empty(0, 5, 2, device="cuda")
    assert S().pairs(X, X, 1).shape == (0,)
    Y = to_dev(np.zeros((3, 5, 2)))
    assert S().gram(X, Y, 1).shape == (0, 3)


def test_two_point_paths_closed_form():
    # one coarse cell at dyadic order 1: k = 1 + G + 3G^2/16 + G^3/128
    rng = np.random.default_rng(3)
    a = rng.normal(size=(50, 3)) * 0.7
    b = rng.normal(size=(50, 3)) * 0.7
    X = np.stack([np.zeros_like(a), a], 1)
    Y = np.stack([np.zeros_like(b), b], 1)
    G = (a * b).sum(1)
    want = 1 + G + 3 * G ** 2 / 16 + G ** 3 / 128
    got = S().pairs(to_dev(X, torch.float64), to_dev(Y, torch.float64), 1).cpu().numpy()
    assert rel_err(got, want) <= F64_TOL


@pytest.mark.parametrize("lam", [5, 6, 8])
def test_high_dyadic_orders(lam):
    X32, X64 = inputs.f32(inputs.random_paths(400, 3, 6, 3))
    Y32, Y64 = inputs.f32(inputs.random_paths(401, 3, 5, 3))
    ref = oracle.pairs(X64, Y64, lam)
    got = S().pairs(to_dev(X32), to_dev(Y32), lam).cpu().numpy()
    assert rel_err(got, ref) <= 1e-4   # FP32 at 256x more cells per coarse cell
    got64 = S().pairs(to_dev(X64, torch.float64), to_dev(Y64, torch.float64), lam).cpu().numpy()
    assert rel_err(got64, ref) <= F64_TOL


def test_nan_propagates():
    X = np.random.default_rng(5).normal(size=(3, 20, 4)) * 0.2
    Y = np.random.default_rng(6).normal(size=(3, 20, 4)) * 0.2
    X[1, 7, 2] = np.nan
    got = S().pairs(to_dev(X), to_dev(Y), 2).cpu().numpy()
    assert np.isnan(got[1]) and np.isfinite(got[[0, 2]]).all()


def test_varlen_pairs_match_oracle():
    w = inputs.uneven_pairs(B=64, lo=8, hi=120, d=16)
    lam = w["dyadic_order"]
    X32, X64 = inputs.f32(w["Xp"])
    Y32, Y64 = inputs.f32(w["Yp"])
    ref = oracle.pairs_varlen(X64, w["x_off"], Y64, w["y_off"], lam)
    xo = torch.as_tensor(w["x_off"]).cuda()
    yo = torch.as_tensor(w["y_off"]).cuda()
    got = S().pairs_varlen(to_dev(X32), xo, to_dev(Y32), yo, lam, max_len=120).cpu().numpy()
    assert rel_err(got, ref) <= F32_TOL
    got64 = S().pairs_varlen(to_dev(X64, torch.float64), xo, to_dev(Y64, torch.float64), yo, lam,
                             max_len=120).cpu().numpy()
    assert rel_err(got64, ref) <= F64_TOL


def test_chain_requested_but_unsupported_is_an_error():
    # dyadic order 4: neither the chained kernel nor the strip path has an instance
    X = to_dev(np.zeros((2, 5, 40)))
    with pytest.raises(S().SigkError):
        S().pairs(X, X, 4, rec=S().REC_CHAIN)
