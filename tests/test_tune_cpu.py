"""Host logic of the autotuner (tune.py) with the timing stubbed out: it
times every candidate, re-times the three leaders with three times the
repetitions and keeps the fastest, tries the double-float redo, the
first-level kernel and the partial FP64 redo on each FP32 leader, then the
placement knobs one at a time, and caches the choice per device, precision,
input kind and size bucket."""
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
        knob = sum(speed.get((k, cfg[k]), 0.0) for k in ("esc_in_pass", "refine_in_pass",
                                                          "tail_warp_items") if k in cfg)
        return speed.get(key, 1.0) + knob + (0.0 if reps == 20 else 0.001)

    monkeypatch.setattr(tune, "time_config", fake_time)
    monkeypatch.setattr(tune, "_key", lambda p, k, n: "dev|%s|%s|%d" % (p, k, n))
    return calls, speed


def test_fastest_leader_is_kept_and_cached(stub, tmp_path):
    calls, speed = stub
    speed.update({(0, 64): 0.50, (hv.OPT_PREFETCH, 128): 0.40, (0, 256): 0.45})
    cache = str(tmp_path / "t.json")
    best = tune.best_config("fp32", "indexed", 1000, None, cache=cache, reps=20)
    defaults = dict(esc_in_pass=4096, refine_in_pass=512, tail_warp_items=8)
    assert best == dict(options=hv.OPT_PREFETCH, bulk_threads=128, **defaults)
    n_cand = len(tune.candidates("fp32"))
    n_knob = sum(len(v) - 1 for _, v in tune.KNOBS["fp32"])
    # all, the three leaders again, the three option trials on each, the knob
    # trials, the three next combinations again with the knobs found
    assert len(calls) == n_cand + 3 + 3 * 3 + n_knob + 3
    assert all(r == 60 for _, r in calls[n_cand:])
    assert calls[n_cand + 3][0] == {"options": hv.OPT_PREFETCH | hv.OPT_DFREDO, "bulk_threads": 128}
    assert calls[n_cand + 4][0] == {"options": hv.OPT_PREFETCH | hv.OPT_LEVEL1, "bulk_threads": 128}
    assert calls[n_cand + 5][0] == {"options": hv.OPT_PREFETCH | hv.OPT_PARTIAL64,
                                    "bulk_threads": 128}
    # the two redos of the escalation list are never combined (hexval_create
    # refuses that)
    both = hv.OPT_DFREDO | hv.OPT_PARTIAL64
    assert all(c["options"] & both != both for c, _ in calls)
    data = json.load(open(cache))
    assert data["dev|fp32|indexed|1000"]["config"] == best
    calls.clear()
    assert tune.best_config("fp32", "indexed", 1000, None, cache=cache) == best
    assert calls == []  # from the cache


def test_option_on_a_later_leader_can_win(stub, tmp_path):
    """The fastest bulk pass alone (packed pairs) is not the fastest with the
    first-level kernel: the option is tried on every leader."""
    calls, speed = stub
    speed.update({(hv.OPT_PAIR32, 64): 0.40, (0, 64): 0.41, (0, 128): 0.42,
                  (hv.OPT_PAIR32 | hv.OPT_LEVEL1, 64): 0.35, (hv.OPT_LEVEL1, 64): 0.30})
    best = tune.best_config("fp32", "soa", 10, None, cache=str(tmp_path / "c.json"))
    assert (best["options"], best["bulk_threads"]) == (hv.OPT_LEVEL1, 64)


def test_options_rechecked_with_the_knobs_found(stub, tmp_path):
    """A combination that loses under the default knobs but wins with the
    knobs found is taken."""
    calls, speed = stub
    speed.update({(hv.OPT_PAIR32 | hv.OPT_LEVEL1, 64): 0.30, (hv.OPT_LEVEL1, 64): 0.31,
                  (hv.OPT_PAIR32, 64): 0.40, (0, 64): 0.41,
                  ("esc_in_pass", 0): -0.05})
    real = tune.time_config

    def with_interaction(cfg, *a, **k):
        ms = real(cfg, *a, **k)
        if cfg.get("esc_in_pass") == 0 and cfg["options"] == hv.OPT_LEVEL1:
            ms -= 0.05  # this combination gains more from the knob
        return ms
    tune.time_config = with_interaction
    try:
        best = tune.best_config("fp32", "soa", 10, None, cache=str(tmp_path / "d.json"))
    finally:
        tune.time_config = real
    assert (best["options"], best["esc_in_pass"]) == (hv.OPT_LEVEL1, 0)


def test_redo_kept_when_faster_and_never_for_fp64(stub, tmp_path):
    calls, speed = stub
    speed.update({(0, 64): 0.30, (hv.OPT_DFREDO, 64): 0.20})
    best = tune.best_config("fp32", "soa", 10, None, cache=str(tmp_path / "a.json"))
    assert best["options"] == hv.OPT_DFREDO and best["bulk_threads"] == 64
    calls.clear()
    best64 = tune.best_config("fp64", "soa", 10, None, cache=str(tmp_path / "b.json"))
    assert all(not (c["options"] & (hv.OPT_DFREDO | hv.OPT_PARTIAL64)) for c, _ in calls)
    assert best64["options"] == 0


def test_placement_knobs_one_at_a_time(stub, tmp_path):
    """A knob value is kept when it is faster, and the search goes on from
    it; the FP64 form tries only the tail threshold."""
    calls, speed = stub
    speed.update({(0, 64): 0.30, ("esc_in_pass", 0): -0.05, ("tail_warp_items", 32): -0.02,
                  ("refine_in_pass", 4096): +0.1})
    best = tune.best_config("fp32", "indexed", 10, None, cache=str(tmp_path / "k.json"))
    assert (best["esc_in_pass"], best["refine_in_pass"], best["tail_warp_items"]) == (0, 512, 32)
    assert [c for c, _ in calls if c.get("tail_warp_items") == 32][0]["esc_in_pass"] == 0
    calls.clear()
    best64 = tune.best_config("fp64", "soa", 10, None, cache=str(tmp_path / "k64.json"))
    assert best64["tail_warp_items"] == 32 and "esc_in_pass" not in best64
    assert {c.get("tail_warp_items") for c, _ in calls} >= {2, 32}


def test_candidates_cover_the_launch_space():
    c32, c64 = tune.candidates("fp32"), tune.candidates("fp64")
    assert {c["bulk_threads"] for c in c32} == {64, 128, 256}
    assert {c["options"] for c in c32} == {0, hv.OPT_PREFETCH, hv.OPT_PAIR32}
    assert all(c["options"] == 0 for c in c64)
