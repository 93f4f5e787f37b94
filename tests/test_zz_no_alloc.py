"""sigk_pairs_backward_noalloc: the pairs backward for callers that cannot
allocate device memory at call time.  Such a caller hands all of its device
memory to its own pool at start-up, or runs under a fixed budget, so one more
cudaMalloc would fail or stall it.  Its scratch is a fixed array in the
library's device image instead of a caller workspace.

Called through the C ABI and compared with the oracle's gradient and with
sigk_pairs_backward (which takes a workspace).  Each case makes two calls in
a row with different inputs, so anything the first call left in the shared
array would show in the second.  The near-limit cases give each pair nearly
the whole array, so one thread block walks every pair through the same
scratch slot.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20


def _noalloc(S, lib, X, Y, g, lam):
    B, L, d = X.shape
    M = Y.shape[1]
    st = torch.cuda.current_stream().cuda_stream
    dX = torch.empty_like(X)
    dY = torch.empty_like(Y)
    code = 1 if X.dtype == torch.float64 else 0
    r = lib.sigk_pairs_backward_noalloc(g.data_ptr(), X.data_ptr(), Y.data_ptr(), B, L, M, d, lam,
                                        code, dX.data_ptr(), dY.data_ptr(), st)
    assert r == S.SIGK_OK, lib.sigk_strerror(r)
    torch.cuda.synchronize()
    return dX.cpu().numpy(), dY.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


def _slot_bytes(L, M, lam, es):
    # one pair's scratch: the coefficients and their adjoint, then the K grid
    ni, nj = (L - 1) << lam, (M - 1) << lam
    return (2 * (L - 1) * (M - 1) + (ni + 1) * (nj + 1)) * es


def _check_twice(cases, dtype, tol):
    from paper_2006_14794_gb300 import sigk as S
    lib = S.lib()
    for call, (seed, B, L, M, d, lam) in enumerate(cases):
        X64 = inputs.random_paths(seed, B, L, d, scale=2.0, time_channel=True)
        Y64 = inputs.random_paths(seed + 50, B, M, d, scale=2.0, time_channel=True)
        g64 = np.random.default_rng(seed).normal(size=B)
        if dtype == torch.float32:
            # the oracle runs on the FP32 inputs promoted to FP64
            X64 = X64.astype(np.float32).astype(np.float64)
            Y64 = Y64.astype(np.float32).astype(np.float64)
            g64 = g64.astype(np.float32).astype(np.float64)
        X, Y, g = to_dev(X64, dtype), to_dev(Y64, dtype), to_dev(g64, dtype)
        dX, dY = _noalloc(S, lib, X, Y, g, lam)
        wX, wY = oracle.pairs_grad(X64, Y64, lam, g64)
        assert _rel(dX, wX) <= tol, (call, "vs oracle", _rel(dX, wX))
        assert _rel(dY, wY) <= tol, (call, "vs oracle", _rel(dY, wY))
        rX, rY = S.pairs_backward(g, X, Y, lam)
        assert _rel(dX, rX.cpu().numpy()) <= tol, (call, "vs workspace backward")
        assert _rel(dY, rY.cpu().numpy()) <= tol, (call, "vs workspace backward")


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-4), (torch.float64, 1e-10)])
def test_noalloc_backward_matches_oracle_twice(dtype, tol):
    need_gpu()
    _check_twice([(900, 37, 33, 20, 3, 1), (901, 19, 24, 41, 5, 2)], dtype, tol)


@pytest.mark.parametrize("dtype,tol,L", [(torch.float32, 1e-4, 1400), (torch.float64, 1e-10, 1000)])
def test_noalloc_near_limit_one_block_reuses_its_slot(dtype, tol, L):
    need_gpu()
    es = 8 if dtype == torch.float64 else 4
    slot = _slot_bytes(L, L, 0, es)
    # a pair takes more than half the array: one block, three pairs in turn
    assert SCRATCH_BYTES // 2 < slot <= SCRATCH_BYTES
    _check_twice([(910, 3, L, L, 2, 0), (911, 3, L, L - 7, 3, 0)], dtype, tol)


def test_noalloc_rejects_pairs_beyond_the_scratch():
    need_gpu()
    from paper_2006_14794_gb300 import sigk as S
    lib = S.lib()
    X = torch.zeros(1, 3000, 2, device="cuda")   # one pair: ~(6000 x 6000) floats of grid > 32 MiB
    assert _slot_bytes(3000, 3000, 1, 4) > SCRATCH_BYTES
    g = torch.ones(1, device="cuda")
    r = lib.sigk_pairs_backward_noalloc(g.data_ptr(), X.data_ptr(), X.data_ptr(), 1, 3000, 3000, 2, 1,
                                        0, X.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert r == S.SIGK_EUNSUPPORTED
