"""The autotuner's selection and cache logic with fake timings (no GPU):
median of repeats, one untimed run per candidate, persistence across
instances, invalidation when the candidates change, and a damaged cache."""
import json
import os

import pytest

from paper_1911_11906_gb300 import autotune as A


class FakeClock:
    """measure(c) returns the next value of c's list (and counts calls)."""

    def __init__(self, seq):
        self.seq = {k: list(v) for k, v in seq.items()}
        self.calls = []

    def __call__(self, c):
        self.calls.append(c)
        return self.seq[c].pop(0)


def test_picks_the_smallest_median_after_a_warm_up(tmp_path):
    t = A.Autotuner(str(tmp_path / "c.json"))
    # first value of each list is the untimed warm-up (made huge for 64 to show it is ignored)
    clk = FakeClock({32: [9.0, 2.0, 9.0, 2.1], 64: [99.0, 1.5, 1.6, 50.0]})
    assert t.choose("eig_band_width", {"n_bucket": 26}, (32, 64), clk, reps=3) == 64
    assert clk.calls == [32, 32, 32, 32, 64, 64, 64, 64]
    e = json.load(open(tmp_path / "c.json"))["entries"]
    (key, val), = e.items()
    assert key.startswith("eig_band_width:") and val["best"] == 64
    assert val["seconds"] == {"32": 2.1, "64": 1.6} and val["reps"] == 3


def test_cache_is_reused_and_invalidated(tmp_path):
    path = str(tmp_path / "sub" / "c.json")
    t = A.Autotuner(path)
    t.choose("op", {"a": 1}, (1, 2), FakeClock({1: [0, 1, 1], 2: [0, 2, 2]}), reps=2)
    clk = FakeClock({})
    assert A.Autotuner(path).choose("op", {"a": 1}, (1, 2), clk) == 1 and clk.calls == []
    # other fields: measured again
    clk = FakeClock({1: [0, 3], 2: [0, 1]})
    assert A.Autotuner(path).choose("op", {"a": 2}, (1, 2), clk, reps=1) == 2
    # the cached winner is no longer offered: measured again among the new candidates
    clk = FakeClock({2: [0, 5], 3: [0, 4]})
    assert A.Autotuner(path).choose("op", {"a": 1}, (2, 3), clk, reps=1) == 3
    assert len(json.load(open(path))["entries"]) == 2
    assert not [f for f in os.listdir(os.path.dirname(path)) if f.endswith(".tmp")]


def test_ties_go_to_the_first_candidate_and_bad_input(tmp_path):
    t = A.Autotuner(str(tmp_path / "c.json"))
    assert t.choose("op", {}, (8, 4), FakeClock({8: [0, 1], 4: [0, 1]}), reps=1) == 8
    with pytest.raises(ValueError):
        t.choose("op", {"x": 1}, (), FakeClock({}))


def test_damaged_cache_starts_empty(tmp_path, monkeypatch):
    path = tmp_path / "c.json"
    path.write_text("{not json")
    t = A.Autotuner(str(path))
    assert t.entries == {}
    assert t.choose("op", {}, (1,), FakeClock({1: [0, 1]}), reps=1) == 1
    assert json.load(open(path))["version"] == 1
    monkeypatch.setenv("FRACLAP_AUTOTUNE_CACHE", str(tmp_path / "env.json"))
    assert A.default_cache_path() == str(tmp_path / "env.json")
    assert A.Autotuner().path == str(tmp_path / "env.json")


def test_size_buckets():
    assert A.size_bucket(8810) == A.size_bucket(8192) != A.size_bucket(16384)
    assert A.size_bucket(1) == 0 and A.size_bucket(0) == 0


def test_apply_schedule_sets_every_knob():
    class FakeCtx:
        def __init__(self):
            self.set = {}

        def set_schedule(self, knob, value):
            self.set[knob] = value

    c = FakeCtx()
    A.apply_schedule(c, {"ozaki_group": 8, "ozaki_bits": 7})
    assert c.set == {"ozaki_group": 8, "ozaki_bits": 7}
