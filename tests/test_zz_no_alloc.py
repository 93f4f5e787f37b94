"""sigk_pairs_backward_noalloc: the pairs backward for callers that cannot
allocate device memory at call time (their device memory is all held by their
own pool, or they run under a fixed budget).  Its scratch is a fixed array in
the library's device image instead of a caller workspace.

Called through the C ABI and compared with sigk_pairs_backward (which takes a
workspace) on two calls in a row with different inputs, so that anything left
in the shared array by the first call would show in the second.  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu


def _both(S, lib, X, Y, g, lam, dt):
    B, L, d = X.shape
    M = Y.shape[1]
    st = torch.cuda.current_stream().cuda_stream
    dX = torch.empty_like(X)
    dY = torch.empty_like(Y)
    code = 1 if X.dtype == torch.float64 else 0
    r = lib.sigk_pairs_backward_noalloc(g.data_ptr(), X.data_ptr(), Y.data_ptr(), B, L, M, d, lam,
                                        code, dX.data_ptr(), dY.data_ptr(), st)
    assert r == S.SIGK_OK, lib.sigk_strerror(r)
    rX, rY = S.pairs_backward(g, X, Y, lam)
    torch.cuda.synchronize()
    return dX.cpu().numpy(), dY.cpu().numpy(), rX.cpu().numpy(), rY.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-4), (torch.float64, 1e-10)])
def test_noalloc_backward_matches_workspace_backward_twice(dtype, tol):
    need_gpu()
    from paper_2006_14794_gb300 import sigk as S
    lib = S.lib()
    for call, (seed, B, L, M, d, lam) in enumerate([(900, 37, 33, 20, 3, 1), (901, 19, 24, 41, 5, 2)]):
        X = to_dev(inputs.random_paths(seed, B, L, d, scale=2.0, time_channel=True), dtype)
        Y = to_dev(inputs.random_paths(seed + 50, B, M, d, scale=2.0, time_channel=True), dtype)
        g = to_dev(np.random.default_rng(seed).normal(size=B), dtype)
        dX, dY, rX, rY = _both(S, lib, X, Y, g, lam, dtype)
        assert _rel(dX, rX) <= tol, (call, _rel(dX, rX))
        assert _rel(dY, rY) <= tol, (call, _rel(dY, rY))


def test_noalloc_rejects_pairs_beyond_the_scratch():
    need_gpu()
    from paper_2006_14794_gb300 import sigk as S
    lib = S.lib()
    X = torch.zeros(1, 3000, 2, device="cuda")   # one pair: ~(6000 x 6000) floats of grid > 32 MiB
    g = torch.ones(1, device="cuda")
    r = lib.sigk_pairs_backward_noalloc(g.data_ptr(), X.data_ptr(), X.data_ptr(), 1, 3000, 3000, 2, 1,
                                        0, X.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert r == S.SIGK_EUNSUPPORTED
