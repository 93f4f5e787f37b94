"""The workloads at their full sizes, in the launch configuration the library
picks for them, checked against the oracle on sampled outputs (the oracle
computes them one by one)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    from paper_2006_14794_gb300 import sigk
    sigk.lib()


def S():
    from paper_2006_14794_gb300 import sigk
    return sigk


def test_uneven_pairs_4096_sampled():
    w = inputs.uneven_pairs()
    lam = w["dyadic_order"]
    X32, X64 = inputs.f32(w["Xp"])
    Y32, Y64 = inputs.f32(w["Yp"])
    xo, yo = w["x_off"], w["y_off"]
    got = S().pairs_varlen(to_dev(X32), torch.as_tensor(xo).cuda(), to_dev(Y32),
                           torch.as_tensor(yo).cuda(), lam, max_len=512,
                           check_status=True).cpu().numpy()
    assert np.isfinite(got).all()
    rng = np.random.default_rng(8)
    idx = np.concatenate([rng.integers(0, 4096, size=60), [0, 4095]])
    lens = (xo[1:] - xo[:-1]) * (yo[1:] - yo[:-1])
    idx = np.concatenate([idx, [int(np.argmax(lens)), int(np.argmin(lens))]])
    ref = np.array([oracle.sigkernel(X64[xo[b]:xo[b + 1]], Y64[yo[b]:yo[b + 1]], lam) for b in idx])
    assert rel_err(got[idx], ref) <= 1e-5


@pytest.mark.parametrize("lam", [0, 1])
def test_long_pairs_sampled(lam):
    w = inputs.long_pairs()
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    got = S().pairs(to_dev(X32), to_dev(Y32), lam, check_status=True).cpu().numpy()
    assert np.isfinite(got).all()
    idx = [0, 37, 63]
    ref = oracle.pairs(X64[idx], Y64[idx], lam)
    assert rel_err(got[idx], ref) <= 1e-5
    g64 = S().pairs(to_dev(X64[idx], torch.float64), to_dev(Y64[idx], torch.float64), lam,
                    rec=S().REC_CHAIN, check_status=True).cpu().numpy()
    assert rel_err(g64, ref) <= 1e-11


def test_mmd_workload_full_sampled_gradient():
    w = inputs.mmd_batches()
    lam = w["dyadic_order"]
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    X = to_dev(X32).requires_grad_(True)
    v = S().mmd2_loss(X, to_dev(Y32), lam)
    v.backward()
    g = X.grad.cpu().numpy()
    assert np.isfinite(g).all()
    ref = oracle.mmd2(X64, Y64, lam)
    assert abs(v.item() - ref) <= 1e-5 * max(1.0, abs(ref))
    m = n = 128
    gxx = np.full((1, m), 1.0 / (m * (m - 1)))
    gxy = np.full((1, n), -2.0 / (m * n))
    for i in (0, 77):
        gi = gxx.copy()
        gi[0, i] = 0.0
        a, _ = oracle.gram_grad(X64[i:i + 1], X64, lam, gi, want_dy=False)
        b, _ = oracle.gram_grad(X64[i:i + 1], Y64, lam, gxy, want_dy=False)
        want = 2.0 * a[0] + b[0]
        err = np.max(np.abs(g[i] - want)) / np.max(np.abs(want))
        assert err <= 1e-4, (i, err)
