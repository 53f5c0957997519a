"""The launch-shape autotuner's host logic (no GPU): candidates stay inside
the library's ranges, the coordinate descent finds the fastest value of each
knob on a stand-in target whose sweep time depends on the configuration, and
the cache round-trips."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_1908_04489_gb300 import autotune as A  # noqa: E402
from paper_1908_04489_gb300 import workloads as W  # noqa: E402


def test_candidates_stay_in_range():
    base = A.default_config()
    for slot in range(5):
        for c in A.candidates(base, "u1_threads", slot):
            assert c["u1_threads"][slot] in (1, 2, 4)
            assert c["u1_threads"][slot] <= 1 << slot
    assert {c["search_lanes"] for c in A.candidates(base, "search_lanes")} == {4, 8, 16}
    assert all(1 <= c["defer_blocks"] <= 4096 for c in A.candidates(base, "defer_blocks"))


def test_run_slots_and_key_of_the_batched_workload():
    ps = W.c3()
    slots = A.run_slots(ps)
    assert slots and all(0 <= s <= 4 for s in slots)
    key = A.workload_key(ps)
    assert key.startswith("n<=256|") and "0.01:1201" in key and "0.02:601" in key


class FakeTarget:
    """Sweep time: a bowl over the knobs with its minimum at lanes 4,
    u1 threads 2 on the slots used, 8 deferred blocks."""

    def __init__(self):
        self.cfg = None
        self.clock = 0.0

    def set_launch_config(self, cfg):
        self.cfg = cfg

    def sweep_ms(self):
        c = self.cfg
        lanes = c["search_lanes"] or 8
        t = 1.0 + 0.1 * abs(lanes - 4) / 4
        for v in c["u1_threads"]:
            t += 0.05 * abs((v or 4) - 2)
        t += 0.02 * abs((c["defer_blocks"] or 4) - 8)
        return t


def test_descent_finds_each_knobs_best_value(monkeypatch):
    tgt = FakeTarget()
    monkeypatch.setattr(A, "time_config", lambda target, cfg, stream, sweeps=3, reps=3:
                        (target.set_launch_config(cfg), target.sweep_ms())[1])
    ps = W.c3()[:8]
    best, table = A.tune(tgt, ps, stream=None)
    assert best["search_lanes"] == 4 and best["defer_blocks"] == 8
    for s in A.run_slots(ps):
        assert best["u1_threads"][s] == 2
    assert tgt.cfg == best and len(table) > 3


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "cache.json")
    assert A.lookup("GB300", "k", path) is None
    A.store("GB300", "k", {"search_lanes": 4, "u1_threads": [0, 0, 0, 2, 4],
                           "defer_blocks": 0}, 1.25, path)
    hit = A.lookup("GB300", "k", path)
    assert hit["config"]["search_lanes"] == 4 and hit["ms_per_sweep"] == 1.25
