"""The strip path (persistent strip wavefront with bounded waits, coarse-cell
coefficients formed by their own kernel): parity with the FP64 oracle on long,
uneven and wide pairs, and its failure detection."""
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


@pytest.mark.parametrize("lam,L,M,d", [
    (0, 700, 300, 3),     # 699 rows: two strips, the first with virtual rows
    (1, 400, 520, 8),     # rows refine the longer (second) path
    (2, 150, 160, 4),
    (3, 70, 90, 5),
    (1, 120, 130, 32),    # wide d: no chained instance
    (0, 1600, 40, 2),     # many strips, narrow grid
])
def test_strip_pairs_match_oracle(lam, L, M, d):
    B = 5
    X32, X64 = inputs.f32(inputs.random_paths(1100 + lam, B, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(1200 + lam, B, M, d, time_channel=True))
    ref = oracle.pairs(X64, Y64, lam)
    got = S().pairs(to_dev(X32), to_dev(Y32), lam, check_status=True).cpu().numpy()
    assert rel_err(got, ref) <= 1e-5
    g64 = S().pairs(to_dev(X64, torch.float64), to_dev(Y64, torch.float64), lam, rec=S().REC_CHAIN,
                    check_status=True).cpu().numpy()
    assert rel_err(g64, ref) <= 1e-11


def test_strip_gram_uneven_batches():
    lam = 1
    X32, X64 = inputs.f32(inputs.random_paths(1300, 4, 300, 6, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(1301, 3, 270, 6, time_channel=True))
    ref = oracle.gram(X64, Y64, lam)
    got = S().gram(to_dev(X32), to_dev(Y32), lam, check_status=True).cpu().numpy()
    assert rel_err(got, ref) <= 1e-5
    got = S().gram(to_dev(Y32), to_dev(X32), lam, check_status=True).cpu().numpy()
    assert rel_err(got, ref.T) <= 1e-5


def test_strip_varlen_with_degenerate_pairs():
    rng = np.random.default_rng(14)
    lens_x = [1, 2, 17, 700, 33, 1, 300]
    lens_y = [5, 1, 2, 40, 600, 9, 300]
    d = 3
    xs = [inputs.random_paths(1400 + i, 1, L, d)[0] for i, L in enumerate(lens_x)]
    ys = [inputs.random_paths(1500 + i, 1, M, d)[0] for i, M in enumerate(lens_y)]
    xo = np.concatenate([[0], np.cumsum(lens_x)]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(lens_y)]).astype(np.int64)
    X32, X64 = inputs.f32(np.concatenate(xs))
    Y32, Y64 = inputs.f32(np.concatenate(ys))
    for lam in (0, 1, 2):
        ref = oracle.pairs_varlen(X64, xo, Y64, yo, lam)
        got = S().pairs_varlen(to_dev(X32), torch.as_tensor(xo).cuda(), to_dev(Y32),
                               torch.as_tensor(yo).cuda(), lam, max_len=700,
                               check_status=True).cpu().numpy()
        assert rel_err(got, ref) <= 1e-5
        assert got[0] == 1.0 and got[1] == 1.0 and got[5] == 1.0


def test_injected_fault_is_reported_as_timeout():
    # the first strip of the first pair never publishes its bottom row: the
    # strip below waits out its bounded wait (~1 s) and the call reports
    # SIGK_ETIMEOUT; the context stays usable
    X = to_dev(inputs.random_paths(1600, 2, 1100, 3))
    with pytest.raises(S().SigkError) as e:
        S().pairs(X, X, 0, check_status=True, fault_inject=True)
    assert "timed out" in str(e.value)
    # the next call on the same context is fine
    ref = oracle.pairs(X.double().cpu().numpy(), X.double().cpu().numpy(), 0)
    got = S().pairs(X, X, 0, check_status=True).cpu().numpy()
    assert rel_err(got, ref) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_nan_inputs_pass_through_the_boundary_rows(dtype):
    """A NaN in one pair's path reaches that pair's result and no other, and
    the boundary rows (whose unwritten entries hold an all-ones NaN pattern)
    still hand it on: no wait times out, forward or backward."""
    sigk = S()
    B, L, d = 3, 1100, 3   # 1099 rows: several strips per pair
    X64 = inputs.random_paths(1650, B, L, d)
    Y64 = inputs.random_paths(1651, B, L, d)
    bad = X64.copy()
    bad[1, 300, 1] = np.nan
    X = to_dev(bad, dtype)
    Y = to_dev(Y64, dtype)
    got = sigk.pairs(X, Y, 0, rec=sigk.REC_STRIP, check_status=True).cpu().numpy()
    assert np.isnan(got[1]) and np.all(np.isfinite(got[[0, 2]]))
    keep = np.array([0, 2])
    assert rel_err(got[keep], oracle.pairs(X64[keep], Y64[keep], 0)) <= (1e-5 if dtype == torch.float32 else 1e-11)
    if dtype == torch.float32:
        dX, _ = sigk.pairs_backward(torch.ones(B, device="cuda"), X, Y, 0, rec=sigk.REC_STRIP,
                                    check_status=True)
        assert torch.isnan(dX[1]).any() and torch.isfinite(dX[[0, 2]]).all()


def test_graph_captured_calls_replay_correctly():
    # the uneven-length strip path (memsets, planning, coefficients, sweep) and
    # the chained Gram, each captured once and replayed on new inputs
    w = inputs.uneven_pairs(B=96, lo=20, hi=300, d=16)
    lam = w["dyadic_order"]
    X32, X64 = inputs.f32(w["Xp"])
    Y32, Y64 = inputs.f32(w["Yp"])
    xo = torch.as_tensor(w["x_off"]).cuda()
    yo = torch.as_tensor(w["y_off"]).cuda()
    Xd, Yd = to_dev(X32), to_dev(Y32)
    g = S().graphed(S().pairs_varlen, Xd, xo, Yd, yo, lam, max_len=300)
    ref = oracle.pairs_varlen(X64, w["x_off"], Y64, w["y_off"], lam)
    assert rel_err(g(Xd, xo, Yd, yo).cpu().numpy(), ref) <= 1e-5
    # new values, same shapes
    X2 = Xd * 0.7
    ref2 = oracle.pairs_varlen(X2.double().cpu().numpy(), w["x_off"], Y64, w["y_off"], lam)
    assert rel_err(g(X2, xo, Yd, yo).cpu().numpy(), ref2) <= 1e-5
    A32, A64 = inputs.f32(inputs.random_paths(1700, 9, 60, 8, time_channel=True))
    B32, B64 = inputs.f32(inputs.random_paths(1701, 7, 60, 8, time_channel=True))
    gg = S().graphed(S().gram, to_dev(A32), to_dev(B32), 2)
    assert rel_err(gg(to_dev(A32), to_dev(B32)).cpu().numpy(), oracle.gram(A64, B64, 2)) <= 1e-5


@pytest.mark.parametrize("lam,L,M,d", [
    (0, 700, 300, 64),   # 512-row strips: four 128-row slices per strip
    (1, 400, 520, 40),   # d not a multiple of 8: zero-padded K
    (2, 150, 160, 32),
    (3, 70, 90, 33),     # 64-row strips: half of a 128-row slice
])
def test_strip_tcgen05_coefficients_match_oracle(lam, L, M, d):
    """Coefficients from split-TF32 tcgen05 MMAs (TMEM accumulators) against
    the oracle, and against the FMA and warp-level MMA coefficient paths."""
    sigk = S()
    B = 3
    X32, X64 = inputs.f32(inputs.random_paths(4300 + lam, B, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(4400 + lam, B, M, d, time_channel=True))
    ref = oracle.pairs(X64, Y64, lam)
    outs = {}
    for coef in (sigk.COEF_TC5, sigk.COEF_TC, sigk.COEF_FMA):
        s = sigk.Schedule(sigk.REC_STRIP, 0, coef)
        outs[coef] = sigk.pairs(to_dev(X32), to_dev(Y32), lam, schedule=s, check_status=True).cpu().numpy()
        assert rel_err(outs[coef], ref) <= 1e-5, coef
    assert rel_err(outs[sigk.COEF_TC5], outs[sigk.COEF_FMA]) <= 2e-6


@pytest.mark.parametrize("R,orient,lam", [(4, 1, 1), (8, 2, 0), (8, 1, 2), (16, 2, 1)])
def test_strip_tcgen05_coefficients_on_uneven_pairs(R, orient, lam):
    """The tcgen05 coefficient blocks on packed pairs of uneven lengths: slices
    past a pair's last row, chunks outside its columns (no MMAs, read back as
    zero), 64- to 512-row strips and the last partial diagonal block."""
    sigk = S()
    rng = np.random.default_rng(4700 + R + lam)
    lens_x = np.concatenate([[1, 2, 390, 129], rng.integers(2, 300, size=20)])
    lens_y = np.concatenate([[70, 1, 2, 258], rng.integers(2, 300, size=20)])
    d = 48
    Xp = np.concatenate([inputs.random_paths(4800 + i, 1, int(n), d)[0] for i, n in enumerate(lens_x)])
    Yp = np.concatenate([inputs.random_paths(4900 + i, 1, int(n), d)[0] for i, n in enumerate(lens_y)])
    xo = np.concatenate([[0], np.cumsum(lens_x)]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(lens_y)]).astype(np.int64)
    X32, X64 = inputs.f32(Xp)
    Y32, Y64 = inputs.f32(Yp)
    ref = oracle.pairs_varlen(X64, xo, Y64, yo, lam)
    outs = {}
    for coef in (sigk.COEF_TC5, sigk.COEF_FMA):
        s = sigk.Schedule(sigk.REC_STRIP, R, coef, orient)
        outs[coef] = sigk.pairs_varlen(to_dev(X32), torch.as_tensor(xo).cuda(), to_dev(Y32),
                                       torch.as_tensor(yo).cuda(), lam, int(max(lens_x.max(), lens_y.max())),
                                       schedule=s, check_status=True).cpu().numpy()
        assert rel_err(outs[coef], ref) <= 1e-5, coef
    assert rel_err(outs[sigk.COEF_TC5], outs[sigk.COEF_FMA]) <= 2e-6


@pytest.mark.parametrize("R,orient,lam", [(4, 1, 1), (4, 2, 0), (8, 1, 2), (8, 2, 1), (16, 2, 3)])
def test_strip_heights_and_orientations_on_uneven_pairs(R, orient, lam):
    """128-, 256- and 512-row strips, rows on the longer or the shorter path,
    on packed pairs of uneven lengths (degenerate ones included)."""
    sigk = S()
    rng = np.random.default_rng(45 + R + lam)
    lens_x = np.concatenate([[1, 2, 300], rng.integers(2, 260, size=60)])
    lens_y = np.concatenate([[50, 1, 2], rng.integers(2, 260, size=60)])
    d = 6
    Xp = np.concatenate([inputs.random_paths(4500 + i, 1, int(n), d)[0] for i, n in enumerate(lens_x)])
    Yp = np.concatenate([inputs.random_paths(4600 + i, 1, int(n), d)[0] for i, n in enumerate(lens_y)])
    xo = np.concatenate([[0], np.cumsum(lens_x)]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(lens_y)]).astype(np.int64)
    X32, X64 = inputs.f32(Xp)
    Y32, Y64 = inputs.f32(Yp)
    ref = oracle.pairs_varlen(X64, xo, Y64, yo, lam)
    s = sigk.Schedule(sigk.REC_STRIP, R, sigk.COEF_FMA, orient)
    got = sigk.pairs_varlen(to_dev(X32), torch.as_tensor(xo).cuda(), to_dev(Y32), torch.as_tensor(yo).cuda(),
                            lam, int(max(lens_x.max(), lens_y.max())), schedule=s, check_status=True)
    assert rel_err(got.cpu().numpy(), ref) <= 1e-5


def test_strip_height_without_instance_is_refused():
    sigk = S()
    X = to_dev(inputs.random_paths(4700, 2, 600, 4, time_channel=True))
    with pytest.raises(sigk.SigkError) as ei:   # 4 rows per lane need dyadic order <= 1
        sigk.pairs(X, X, 2, schedule=sigk.Schedule(sigk.REC_STRIP, 4, 0))
    assert ei.value.status == sigk.SIGK_EUNSUPPORTED
