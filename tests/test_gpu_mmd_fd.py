"""The MMD^2 loss's gradient on the full differentiation workload (128 vs 128
paths, L = 256, d = 32, dyadic order 1) against central finite differences of
the library's FP64 MMD^2 at h = 1e-6: 256 seeded coordinates of X and 4
random directions.

The gradient under test is the FP32 adjoint (the band-form reverse sweep
behind mmd2_loss's autograd function).  The differences are taken in FP64 on
the GPU.  For a coordinate X_i[t, c], only the Gram entries with path i in
them change: k(x_i, x_j) for j != i (Kxx is symmetric, so each enters the
U-statistic twice) and k(x_i, y_j).  The difference of MMD^2 is therefore
  2/(m(m-1)) sum_{j!=i} [k(x_i+, x_j) - k(x_i-, x_j)] - 2/(mn) sum_j [k(x_i+, y_j) - k(x_i-, y_j)],
which equals the difference of the whole loss in exact arithmetic and does
not carry the rounding of the unchanged terms.  The directions perturb every
coordinate, so there the whole FP64 MMD^2 is evaluated twice per direction.
Each difference is compared with g . (X+ - X-), the exact step taken."""
import numpy as np
import pytest
import torch

from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu

H = 1e-6
TOL = 1e-4


def _S():
    from paper_2006_14794_gb300 import sigk
    return sigk


@pytest.fixture(scope="module")
def workload():
    need_gpu()
    S = _S()
    S.lib()
    w = inputs.mmd_batches()
    lam = w["dyadic_order"]
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    X = to_dev(X32).requires_grad_(True)
    v = S.mmd2_loss(X, to_dev(Y32), lam)
    v.backward()
    g = X.grad.double().cpu().numpy()
    assert np.isfinite(g).all()
    return dict(lam=lam, X64=X64, Y64=Y64, g=g)


def test_mmd_gradient_vs_central_differences_on_256_coordinates(workload):
    S = _S()
    lam, X64, Y64, g = workload["lam"], workload["X64"], workload["Y64"], workload["g"]
    m, L, d = X64.shape
    n = Y64.shape[0]
    rng = np.random.default_rng(2006_0444)
    coords = np.stack([rng.integers(0, m, 256), rng.integers(0, L, 256), rng.integers(0, d, 256)], 1)
    Xd = to_dev(X64, torch.float64)
    Yd = to_dev(Y64, torch.float64)
    w = torch.tensor([2.0 / (m * (m - 1))] * (m - 1) + [-2.0 / (m * n)] * n, dtype=torch.float64,
                     device="cuda")
    fd_diff = np.zeros(len(coords))    # MMD^2(X+) - MMD^2(X-)
    step = np.zeros(len(coords))       # (X+ - X-) at the coordinate
    for chunk in np.array_split(np.arange(len(coords)), 16):
        A, B = [], []
        for q in chunk:
            i, t, c = (int(v) for v in coords[q])
            partners = torch.cat([Xd[torch.arange(m, device="cuda") != i], Yd])
            xp, xm = Xd[i].clone(), Xd[i].clone()
            xp[t, c] += H
            xm[t, c] -= H
            step[q] = float(xp[t, c] - xm[t, c])
            for xs in (xp, xm):
                A.append(xs.expand(partners.shape[0], -1, -1))
                B.append(partners)
        k = S.pairs(torch.cat(A).contiguous(), torch.cat(B).contiguous(), lam, check_status=True)
        k = k.view(len(chunk), 2, m - 1 + n)
        fd_diff[chunk] = ((k[:, 0, :] - k[:, 1, :]) * w).sum(1).cpu().numpy()
    want = fd_diff
    got = g[coords[:, 0], coords[:, 1], coords[:, 2]] * step
    err = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    assert err <= TOL, err


def test_mmd_gradient_vs_central_differences_in_4_random_directions(workload):
    """Directions v ~ N(0, I) over all of X.  A directional derivative g . v
    can cancel to far below its typical size, so each error is measured
    against that typical size: for v ~ N(0, I), g . v has standard deviation
    |g|_2, and the difference of the loss over the step 2hv has 2h|g|_2."""
    S = _S()
    lam, X64, Y64, g = workload["lam"], workload["X64"], workload["Y64"], workload["g"]
    rng = np.random.default_rng(2006_0445)
    Yd = to_dev(Y64, torch.float64)
    scale = 2.0 * H * float(np.linalg.norm(g))
    rows = []
    for k in range(4):
        V = rng.standard_normal(X64.shape)
        Xp = X64 + H * V
        Xm = X64 - H * V
        with torch.no_grad():
            fp = S.mmd2_loss(to_dev(Xp, torch.float64), Yd, lam).item()
            fm = S.mmd2_loss(to_dev(Xm, torch.float64), Yd, lam).item()
        want = fp - fm
        got = float(np.sum(g * (Xp - Xm)))
        rows.append((k, got, want, abs(got - want) / scale))
    print("directions (k, g.dX, MMD^2(X+) - MMD^2(X-), error / (2h |g|_2)):", rows)
    for k, got, want, err in rows:
        assert err <= TOL, (k, got, want, err)
