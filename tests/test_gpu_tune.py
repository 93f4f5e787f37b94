"""Every schedule (rec, rows_per_lane, coef_path) solves the same scheme: each
one matches the FP64 oracle, and the tuner's choice does too."""
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


@pytest.fixture()
def cache(tmp_path, monkeypatch):
    from paper_2006_14794_gb300 import tune
    monkeypatch.setenv("SIGK_TUNE_CACHE", str(tmp_path / "schedules.json"))
    tune.clear_memory_cache()
    yield tmp_path / "schedules.json"
    tune.clear_memory_cache()


def _S():
    from paper_2006_14794_gb300 import sigk
    return sigk


@pytest.mark.parametrize("lam,L,d", [(1, 33, 4), (0, 200, 8), (2, 40, 40)])
def test_every_schedule_matches_oracle(lam, L, d):
    from paper_2006_14794_gb300 import tune
    sigk = _S()
    X32, X64 = inputs.f32(inputs.random_paths(2100 + lam, 6, L, d, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(2200 + lam, 5, L, d, time_channel=True))
    ref = oracle.gram(X64, Y64, lam)
    ran = 0
    for s in tune.candidates("gram", torch.float32):
        try:
            got = sigk.gram(to_dev(X32), to_dev(Y32), lam, schedule=s, check_status=True)
        except sigk.SigkError as e:
            # only a row count without an instance for this shape may refuse
            assert e.status == sigk.SIGK_EUNSUPPORTED and s.rows_per_lane != 0, s
            continue
        assert rel_err(got.cpu().numpy(), ref) <= 1e-5, s
        ran += 1
    assert ran >= 3
    for s in tune.candidates("gram", torch.float64):
        got = sigk.gram(to_dev(X64, torch.float64), to_dev(Y64, torch.float64), lam, schedule=s,
                        check_status=True)
        assert rel_err(got.cpu().numpy(), ref) <= 1e-11, s


def test_chained_row_count_without_instance_is_refused():
    sigk = _S()
    X = to_dev(inputs.random_paths(2300, 2, 129, 3, time_channel=True))
    # 256 refined rows do not fit 32 lanes x 4 rows
    with pytest.raises(sigk.SigkError) as ei:
        sigk.pairs(X, X, 1, schedule=sigk.Schedule(sigk.REC_CHAIN, 4, 0))
    assert ei.value.status == sigk.SIGK_EUNSUPPORTED


def test_tuned_gram_and_cache(cache):
    from paper_2006_14794_gb300 import tune
    sigk = _S()
    lam = 1
    X32, X64 = inputs.f32(inputs.random_paths(2400, 8, 65, 4, time_channel=True))
    ref = oracle.gram(X64, X64, lam)
    Xd = to_dev(X32)
    got = sigk.gram(Xd, Xd, lam, schedule="tuned").cpu().numpy()
    assert rel_err(got, ref) <= 1e-5
    assert cache.exists()
    s = tune.lookup("gram", Xd, Xd, lam)
    assert s in tune.candidates("gram", torch.float32)
    # a fresh process-level cache reads the same choice back from the file
    tune.clear_memory_cache()
    assert tune.lookup("gram", Xd, Xd, lam) == s


def test_tuned_varlen_matches_oracle(cache):
    sigk = _S()
    rng = np.random.default_rng(25)
    lx = rng.integers(2, 300, size=40)
    ly = rng.integers(2, 300, size=40)
    d, lam = 16, 1
    Xp = np.concatenate([inputs.random_paths(2500 + i, 1, int(n), d)[0] for i, n in enumerate(lx)])
    Yp = np.concatenate([inputs.random_paths(2600 + i, 1, int(n), d)[0] for i, n in enumerate(ly)])
    xo = np.concatenate([[0], np.cumsum(lx)]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(ly)]).astype(np.int64)
    X32, X64 = inputs.f32(Xp)
    Y32, Y64 = inputs.f32(Yp)
    ref = oracle.pairs_varlen(X64, xo, Y64, yo, lam)
    got = sigk.pairs_varlen(to_dev(X32), torch.as_tensor(xo).cuda(), to_dev(Y32),
                            torch.as_tensor(yo).cuda(), lam, int(max(lx.max(), ly.max())),
                            schedule="tuned", check_status=True).cpu().numpy()
    assert rel_err(got, ref) <= 1e-5


@pytest.mark.parametrize("coef", [1, 2])
def test_backward_coefficient_paths_match_oracle(coef):
    sigk = _S()
    lam = 1
    X32, X64 = inputs.f32(inputs.random_paths(2700, 3, 90, 40, time_channel=True))
    Y32, Y64 = inputs.f32(inputs.random_paths(2701, 3, 70, 40, time_channel=True))
    g = np.array([1.0, -0.5, 2.0])
    rdx, rdy = oracle.pairs_grad(X64, Y64, lam, g)
    s = sigk.Schedule(sigk.REC_STRIP, 0, coef)
    dX, dY = sigk.pairs_backward(torch.as_tensor(g).cuda(), to_dev(X32), to_dev(Y32), lam, schedule=s)
    scale_x = np.abs(rdx).max()
    scale_y = np.abs(rdy).max()
    assert np.abs(dX.cpu().numpy() - rdx).max() / scale_x <= 1e-4
    assert np.abs(dY.cpu().numpy() - rdy).max() / scale_y <= 1e-4
