"""Host logic of the schedule tuner: candidate lists, the choice among timed
candidates, and the cache file (no GPU needed)."""
import json

import pytest
import torch

from paper_2006_14794_gb300 import sigk, tune
from paper_2006_14794_gb300.sigk import COEF_FMA, COEF_TC, REC_CHAIN, REC_PLAIN, REC_STRIP, Schedule


def test_candidates_cover_every_path():
    c32 = tune.candidates("gram", torch.float32)
    assert {s.rows_per_lane for s in c32 if s.rec == REC_CHAIN} == {4, 8, 16}
    assert {s.rows_per_lane for s in c32 if s.rec == sigk.REC_BAND} == {4, 8, 16}
    assert Schedule(REC_STRIP, 16, COEF_TC, 1) in c32 and Schedule(REC_STRIP, 4, COEF_FMA, 2) in c32
    assert Schedule(REC_STRIP, 8, sigk.COEF_TC5, 1) in c32
    assert c32[-1].rec == REC_PLAIN
    c64 = tune.candidates("pairs", torch.float64)
    assert all(s.rec not in (REC_CHAIN, sigk.REC_BAND) and s.coef_path != COEF_TC for s in c64)
    cv = tune.candidates("pairs_varlen", torch.float32)
    # uneven lengths: the warp stacks and the band form plan their own heights
    assert [s for s in cv if s.rec == REC_CHAIN] == [Schedule(REC_CHAIN, 0, 0)]
    assert [s for s in cv if s.rec == sigk.REC_BAND] == [Schedule(sigk.REC_BAND, 0, 0)]
    assert all(s.rec not in (REC_CHAIN, sigk.REC_BAND) for s in tune.candidates("pairs_varlen", torch.float64))
    assert all(s.rec != sigk.REC_BAND for s in tune.candidates("pairs_varlen", torch.float64))


def test_pick_takes_the_fastest_that_ran():
    ref = torch.tensor([1.0, 2.0, 3.0])
    res = [(Schedule(REC_CHAIN, 4, 0), None, None),            # no instance
           (Schedule(REC_CHAIN, 8, 0), 2.0, ref.clone()),
           (Schedule(REC_STRIP, 16, COEF_TC, 2), 1.5, ref * (1 + 1e-6)),
           (Schedule(REC_PLAIN, 0, 0), 9.0, ref.clone())]
    s, ms = tune.pick(res, 1e-4)
    assert s == Schedule(REC_STRIP, 16, COEF_TC, 2) and ms == 1.5


def test_pick_rejects_disagreeing_schedules():
    ref = torch.tensor([1.0, 2.0])
    res = [(Schedule(REC_CHAIN, 8, 0), 2.0, ref), (Schedule(REC_PLAIN, 0, 0), 1.0, ref * 1.01)]
    with pytest.raises(sigk.SigkError):
        tune.pick(res, 1e-4)
    with pytest.raises(sigk.SigkError):
        tune.pick([(Schedule(REC_CHAIN, 8, 0), None, None)], 1e-4)


def test_cache_file_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "schedules.json"
    monkeypatch.setenv("SIGK_TUNE_CACHE", str(path))
    tune._store("k1", Schedule(REC_STRIP, 8, COEF_FMA, 2), 1.25)
    tune._store("k2", Schedule(REC_CHAIN, 16, 0), 0.5)
    d = json.loads(path.read_text())
    assert d["k1"] == [REC_STRIP, 8, COEF_FMA, 2, 1.25] and d["k2"] == [REC_CHAIN, 16, 0, 0, 0.5]
    assert tune._load() == d
    path.write_text("not json")
    assert tune._load() == {}
