"""The solution surface on the sample grid (sigk_pairs_surface) through the C
ABI against the FP64 oracle: the band sweep's and the chained sweep's surface
instances for every (rows per lane, dyadic order) family, both orientations,
pair turnovers inside a warp's chain, the plain sweep (f32 and f64, long
pairs), both variants, and the degenerate and refused cases."""
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


@pytest.mark.parametrize("R,lam,L,M,d", [
    (16, 2, 128, 128, 8),    # the bench shape
    (16, 1, 200, 150, 24),   # L > M: rows refine Y, the surface is transposed back
    (8, 0, 230, 256, 5),     # every refined node is a sample-grid node
    (8, 1, 100, 90, 17),
    (16, 3, 40, 61, 3),
    (4, 1, 60, 70, 33),
])
def test_band_surface_matches_oracle(R, lam, L, M, d):
    sigk = S()
    B = 23   # several pairs per warp: turnovers inside the chain
    X32, X64 = inputs.f32(inputs.random_paths(7100 + R + lam, B, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(7200 + R + lam, B, M, d, time_channel=True))
    rk, rs = oracle.pairs_surface(X64, Y64, lam)
    k, surf = sigk.pairs_surface(to_dev(X32), to_dev(Y32), lam,
                                 schedule=sigk.Schedule(sigk.REC_BAND, R, 0))
    surf = surf.cpu().numpy()
    assert surf.shape == (B, L, M)
    assert rel_err(surf, rs) <= F32_TOL
    assert rel_err(k.cpu().numpy(), rk) <= F32_TOL
    np.testing.assert_array_equal(surf[:, :, -1][:, -1], k.cpu().numpy())
    assert np.all(surf[:, 0, :] == 1.0) and np.all(surf[:, :, 0] == 1.0)


@pytest.mark.parametrize("R,lam,L,M,d", [
    (16, 2, 128, 128, 8),    # the bench shape
    (16, 1, 200, 150, 4),    # L > M: rows refine Y, the surface is transposed back
    (8, 0, 230, 256, 5),     # every refined node is a sample-grid node
    (8, 2, 60, 50, 13),      # four channel quads
    (16, 3, 40, 61, 3),
    (4, 1, 60, 70, 16),
])
def test_chain_surface_matches_oracle(R, lam, L, M, d):
    # the chained sweep (coefficients formed inline) writes the nodes' band
    # layout, which the surface unpack reads
    sigk = S()
    B = 23   # several pairs per warp: turnovers inside the chain
    X32, X64 = inputs.f32(inputs.random_paths(7700 + R + lam, B, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(7800 + R + lam, B, M, d, time_channel=True))
    rk, rs = oracle.pairs_surface(X64, Y64, lam)
    k, surf = sigk.pairs_surface(to_dev(X32), to_dev(Y32), lam,
                                 schedule=sigk.Schedule(sigk.REC_CHAIN, R, 0))
    surf = surf.cpu().numpy()
    assert surf.shape == (B, L, M)
    assert rel_err(surf, rs) <= F32_TOL
    assert rel_err(k.cpu().numpy(), rk) <= F32_TOL
    np.testing.assert_array_equal(surf[:, :, -1][:, -1], k.cpu().numpy())
    assert np.all(surf[:, 0, :] == 1.0) and np.all(surf[:, :, 0] == 1.0)
    if R == 16 and lam == 2:
        # AUTO takes the chained surface: the same bits
        k2, s2 = sigk.pairs_surface(to_dev(X32), to_dev(Y32), lam)
        np.testing.assert_array_equal(s2.cpu().numpy(), surf)


@pytest.mark.parametrize("dtype,L,M,lam", [(torch.float32, 50, 70, 1), (torch.float64, 50, 70, 1),
                                           (torch.float32, 700, 40, 0)])   # 699 rows: no band
def test_plain_surface_matches_oracle(dtype, L, M, lam):
    sigk = S()
    B, d = 6, 4
    X32, X64 = inputs.f32(inputs.random_paths(7300 + L, B, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(7400 + M, B, M, d, time_channel=True))
    rk, rs = oracle.pairs_surface(X64, Y64, lam)
    X = to_dev(X32 if dtype == torch.float32 else X64, dtype)
    Y = to_dev(Y32 if dtype == torch.float32 else Y64, dtype)
    rec = sigk.REC_PLAIN if L < 700 else sigk.REC_AUTO
    k, surf = sigk.pairs_surface(X, Y, lam, rec=rec)
    tol = F32_TOL if dtype == torch.float32 else F64_TOL
    assert rel_err(surf.cpu().numpy(), rs) <= tol
    assert rel_err(k.cpu().numpy(), rk) <= tol


@pytest.mark.parametrize("kw", [dict(scheme="implicit"), dict(static_kernel="rbf", sigma=0.9),
                                dict(scheme="implicit", static_kernel="rbf", sigma=1.3)])
def test_surface_variants(kw):
    sigk = S()
    B, L, M, d, lam = 9, 64, 80, 6, 1
    X32, X64 = inputs.f32(inputs.random_paths(7500, B, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(7501, B, M, d, time_channel=True))
    rk, rs = oracle.pairs_surface(X64, Y64, lam, **kw)
    k, surf = sigk.pairs_surface(to_dev(X32), to_dev(Y32), lam, variant=sigk.Variant(**kw))
    assert rel_err(surf.cpu().numpy(), rs) <= F32_TOL
    assert rel_err(k.cpu().numpy(), rk) <= F32_TOL


def test_surface_degenerate_and_refused():
    sigk = S()
    X = to_dev(inputs.random_paths(7600, 3, 1, 4))   # single points: k = 1 everywhere
    Y = to_dev(inputs.random_paths(7601, 3, 9, 4))
    k, surf = sigk.pairs_surface(X, Y, 2)
    assert torch.all(k == 1) and torch.all(surf == 1) and surf.shape == (3, 1, 9)
    Z = to_dev(inputs.random_paths(7602, 3, 9, 4))
    with pytest.raises(sigk.SigkError) as ei:
        sigk.pairs_surface(Z, Z, 1, rec=sigk.REC_STRIP)
    assert ei.value.status == sigk.SIGK_EUNSUPPORTED
    k0, s0 = sigk.pairs_surface(Z[:0], Z[:0], 1)
    assert k0.numel() == 0 and s0.numel() == 0
