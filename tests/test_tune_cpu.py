"""Host logic of the autotuner (tune.py) with the timing stubbed out: it
times every candidate, re-times the three leaders with three times the
repetitions and keeps the fastest, tries the double-float redo on the FP32
winner only, and caches the choice per device, precision, input kind and
size bucket."""
import json

import pytest

from paper_1706_01613_gb300 import hexval as hv
from paper_1706_01613_gb300 import tune


@pytest.fixture
def stub(monkeypatch):
    calls = []
    speed = {}

    def fake_time(cfg, precision, kind, dev_inputs, reps=20, **caps):
        calls.append((dict(cfg), reps))
        key = (cfg["options"], cfg["bulk_threads"])
        return speed.get(key, 1.0) + (0.0 if reps == 20 else 0.001)

    monkeypatch.setattr(tune, "time_config", fake_time)
    monkeypatch.setattr(tune, "_key", lambda p, k, n: "dev|%s|%s|%d" % (p, k, n))
    return calls, speed


def test_fastest_leader_is_kept_and_cached(stub, tmp_path):
    calls, speed = stub
    speed.update({(0, 64): 0.50, (hv.OPT_PREFETCH, 128): 0.40, (0, 256): 0.45})
    cache = str(tmp_path / "t.json")
    best = tune.best_config("fp32", "indexed", 1000, None, cache=cache, reps=20)
    assert best == {"options": hv.OPT_PREFETCH, "bulk_threads": 128}
    n_cand = len(tune.candidates("fp32"))
    assert len(calls) == n_cand + 3 + 1  # all, the three leaders again, the redo trial
    assert [r for _, r in calls[n_cand:]] == [60, 60, 60, 60]
    assert calls[-1][0] == {"options": hv.OPT_PREFETCH | hv.OPT_DFREDO, "bulk_threads": 128}
    data = json.load(open(cache))
    assert data["dev|fp32|indexed|1000"]["config"] == best
    calls.clear()
    assert tune.best_config("fp32", "indexed", 1000, None, cache=cache) == best
    assert calls == []  # from the cache


def test_redo_kept_when_faster_and_never_for_fp64(stub, tmp_path):
    calls, speed = stub
    speed.update({(0, 64): 0.30, (hv.OPT_DFREDO, 64): 0.20})
    best = tune.best_config("fp32", "soa", 10, None, cache=str(tmp_path / "a.json"))
    assert best == {"options": hv.OPT_DFREDO, "bulk_threads": 64}
    calls.clear()
    best64 = tune.best_config("fp64", "soa", 10, None, cache=str(tmp_path / "b.json"))
    assert all(not (c["options"] & hv.OPT_DFREDO) for c, _ in calls)
    assert best64["options"] == 0


def test_candidates_cover_the_launch_space():
    c32, c64 = tune.candidates("fp32"), tune.candidates("fp64")
    assert {c["bulk_threads"] for c in c32} == {64, 128, 256}
    assert {c["options"] for c in c32} == {0, hv.OPT_PREFETCH, hv.OPT_PAIR32}
    assert all(c["options"] == 0 for c in c64)
