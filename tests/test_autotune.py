"""Autotuner host logic (no GPU): size classes, choice of the fastest
candidate, persistence, and refusal of a candidate that changes the count."""
import json

import pytest

from paper_1804_06926_gb300 import autotune


def test_size_class_groups_by_powers_of_two():
    assert autotune.size_class(1024, 16384) == autotune.size_class(1500, 20000)
    assert autotune.size_class(1024, 16384) != autotune.size_class(4096, 16384)
    assert autotune.size_class(1024, 16384, 4096) != autotune.size_class(1024, 16384)


def test_picks_fastest_and_persists(tmp_path):
    path = str(tmp_path / "cache.json")
    t = autotune.Autotuner(path, device_name="fake")
    speed = {"a": 5.0, "b": 2.0, "c": 3.0}
    res = t.tune("cls", lambda cfg: (speed[cfg["k"]], 42), [{"k": "a"}, {"k": "b"}, {"k": "c"}], reps=1)
    assert res.best == {"k": "b"}
    data = json.load(open(path))
    assert data["fake|cls"]["best"] == {"k": "b"}
    # a new tuner reads the cache and does not re-run
    t2 = autotune.Autotuner(path, device_name="fake")
    calls = []
    res2 = t2.tune("cls", lambda cfg: calls.append(cfg) or (1.0, 42), [{"k": "z"}])
    assert res2.best == {"k": "b"} and not calls
    # force re-measures
    res3 = t2.tune("cls", lambda cfg: (1.0, 42), [{"k": "z"}], force=True)
    assert res3.best == {"k": "z"}


def test_rejects_candidate_changing_the_result(tmp_path):
    t = autotune.Autotuner(str(tmp_path / "c.json"), device_name="fake")
    with pytest.raises(RuntimeError):
        t.tune("cls", lambda cfg: (1.0, cfg["T"]), [{"T": 1}, {"T": 2}], reps=1)


def test_greedy_merge_of_winning_knobs(tmp_path):
    """Stage two merges the candidates that beat the default into the
    fastest one, one at a time, and keeps a merge only when it is faster."""
    t = autotune.Autotuner(str(tmp_path / "c.json"), device_name="fake")
    cost = {"a": -3.0, "b": -2.0, "c": +1.0, "d": -1.0}

    def run(cfg):  # additive costs, except that d slows down any merge holding a
        ms = 10.0 + sum(cost[k] for k in cfg)
        if "a" in cfg and "d" in cfg:
            ms += 5.0
        return ms, 7

    cands = [{}, {"a": 1}, {"b": 1}, {"c": 1}, {"d": 1}, {"a": 2}]
    res = t.tune("cls", run, cands, reps=1)
    assert res.best == {"a": 1, "b": 1}
    tried = [c for c, _ in res.times_ms]
    assert tried[:len(cands)] == cands
    # c never beat the default and {"a": 2} shares a knob with the winner: neither is merged;
    # d is merged in after b, measured slower, and dropped
    assert tried[len(cands):] == [{"a": 1, "b": 1}, {"a": 1, "b": 1, "d": 1}]
    # without the second stage the best single candidate wins
    res1 = t.tune("cls2", run, cands, reps=1, combine=False)
    assert res1.best == {"a": 1} and len(res1.times_ms) == len(cands)
