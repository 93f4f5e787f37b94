"""The support-reduction iteration (Sec. 5.3) through the C ABI against the
oracle's iteration, step for step: the paper's fBM example with the Gram from
sigk_gram, a seeded positive definite Gram with a reduced support, f64 and
f32, and the argument checks."""
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


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, 2 * n)) / np.sqrt(2 * n)
    return A @ A.T + 0.05 * np.eye(n)


@pytest.mark.parametrize("n", [30, 257, 1500])
def test_support_reduction_f64_matches_oracle(n):
    sigk = S()
    K = _spd(n, 500 + n)
    a = np.random.default_rng(501).uniform(0.5, 1.5, size=n) / n
    gamma = 0.5 / np.linalg.eigvalsh(K).max()
    lam = 0.02
    rb, rl = oracle.support_reduction(K, a, a.copy(), gamma, lam, 400)
    b, loss = sigk.support_reduction(to_dev(K, torch.float64), to_dev(a, torch.float64),
                                     to_dev(a, torch.float64), gamma, lam, 400)
    np.testing.assert_allclose(b.cpu().numpy(), rb, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(loss.cpu().numpy(), rl, rtol=1e-10)
    assert rl[-1] < rl[0]   # the loss falls


def test_support_reduction_f32_and_the_fbm_gram():
    sigk = S()
    X, H = inputs.fbm_paths()
    X[:, :, 1] *= 0.5 / np.abs(X[:, :, 1]).max()
    X32, X64 = inputs.f32(X)
    Xd = to_dev(X32)
    K = sigk.gram(Xd, Xd, 3)                      # the Gram on the GPU (f32)
    Kh = K.double().cpu().numpy()
    n = Kh.shape[0]
    a = np.full(n, 1.0 / n)
    gamma = 0.5 / np.abs(np.linalg.eigvalsh(Kh)).max()
    lam = 0.5
    rb, rl = oracle.support_reduction(Kh, a, np.zeros(n), gamma, lam, 1000)
    b, loss = sigk.support_reduction(K, to_dev(a), torch.zeros(n, device="cuda"), gamma, lam, 1000)
    np.testing.assert_allclose(b.cpu().numpy(), rb, rtol=1e-4, atol=1e-7)
    np.testing.assert_allclose(loss.cpu().numpy(), rl, rtol=1e-4)
    # and the Gram itself matches the oracle's
    Ko = oracle.gram(X64, X64, 3)
    assert float(np.max(np.abs(Kh - Ko) / np.maximum(np.abs(Ko), 1e-3))) <= 1e-5


def test_support_reduction_argument_checks():
    sigk = S()
    K = torch.eye(4, device="cuda")
    a = torch.ones(4, device="cuda")
    with pytest.raises(sigk.SigkError) as ei:
        sigk.support_reduction(K, a, a, 0.0, 0.1, 10)
    assert ei.value.status == sigk.SIGK_EINVAL
    with pytest.raises(sigk.SigkError) as ei:
        sigk.support_reduction(K, a, a, 0.1, -1.0, 10)
    assert ei.value.status == sigk.SIGK_EINVAL
    big = 17067
    lib = sigk.lib()
    P = torch.zeros(1, device="cuda")
    st = lib.sigk_support_reduction(P.data_ptr(), P.data_ptr(), P.data_ptr(), big, 0.1, 0.1, 1,
                                    sigk.SIGK_F32, None, None)
    assert st == sigk.SIGK_EUNSUPPORTED
    b, loss = sigk.support_reduction(K, a, a, 0.25, 0.0, 0)   # zero steps: beta0, one loss value
    assert torch.equal(b, a) and loss.numel() == 1
