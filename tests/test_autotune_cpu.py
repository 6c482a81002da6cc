"""Host logic of the batched launch's autotuner (paper_2303_01471_gb300/autotune.py)
without a GPU: the candidate set per mix of mesh sizes, the choice of the fastest
measured candidate, and the cache (written once, then read back without timing;
a corrupt cache file is ignored).  The timing itself is replaced by a fake."""
import json
from types import SimpleNamespace

import pytest

from paper_2303_01471_gb300 import autotune, qhd


def fake_sims(*edges):
    return [SimpleNamespace(shape=(e, e), batch=3) for e in edges]


def test_candidates_cover_the_allowed_splits():
    c = autotune.candidates(fake_sims(128, 256))
    subs = sorted({tuple(x.as_dict()["sub"]) for x in c})
    assert subs == [(0, 4, 8), (0, 8, 8)]
    assert sorted({x.min_blocks for x in c}) == [1, 2]
    assert len(c) == 4
    c = autotune.candidates(fake_sims(64, 128))
    assert len(c) == 3 * 2 * 2
    assert all(x.as_dict()["sub"][2] == 0 for x in c)       # no 256^2 context: its slot stays default
    assert len(autotune.candidates(fake_sims(256))) == 2


def test_tuner_keeps_the_fastest_and_caches_it(tmp_path, monkeypatch):
    sims = fake_sims(128, 256)
    calls = []

    def fake_time(s, cfg, T, dt, reps=2):
        calls.append(cfg.as_dict())
        d = cfg.as_dict()
        return 10.0 + d["sub"][1] - 3.0 * d["min_blocks"]    # fastest: sub 4 for 128^2, 2 CTAs per SM

    monkeypatch.setattr(autotune, "time_config", fake_time)
    monkeypatch.setattr(autotune, "cache_key", lambda s: "fake-gpu|152|lib|[(128, 3), (256, 3)]")
    cache = tmp_path / "tune" / "group.json"
    res = autotune.tune_group(sims, cache_file=str(cache))
    assert not res["cached"] and len(calls) == 4
    assert res["config"].as_dict() == {"sub": [0, 4, 8], "min_blocks": 2, "clusters": 0}
    assert [m for m, _ in res["ms"]] == sorted(m for m, _ in res["ms"])
    stored = json.loads(cache.read_text())
    assert list(stored) == ["fake-gpu|152|lib|[(128, 3), (256, 3)]"]

    again = autotune.tune_group(sims, cache_file=str(cache))
    assert again["cached"] and len(calls) == 4                   # read back, nothing timed
    assert again["config"].as_dict() == res["config"].as_dict()

    forced = autotune.tune_group(sims, use_cache=False, cache_file=str(cache))
    assert not forced["cached"] and len(calls) == 8


def test_corrupt_cache_is_ignored(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "time_config", lambda s, cfg, T, dt, reps=2: float(cfg.min_blocks))
    monkeypatch.setattr(autotune, "cache_key", lambda s: "k")
    cache = tmp_path / "group.json"
    cache.write_text("{not json")
    res = autotune.tune_group(fake_sims(256), cache_file=str(cache))
    assert not res["cached"] and res["config"].min_blocks == 1
    assert json.loads(cache.read_text())["k"]["config"]["min_blocks"] == 1


def test_group_config_round_trip():
    c = qhd.GroupConfig.make((2, 4, 8), 2, 36)
    assert c.as_dict() == {"sub": [2, 4, 8], "min_blocks": 2, "clusters": 36}
    with pytest.raises(Exception):
        qhd.GroupConfig.make((2, 4, 8, 16), 1, 0)
