"""Host-side checks of the benchmark's bookkeeping (no GPU): every DRAM-traffic entry that
bench.py may report names a committed profile summary, and that summary records the source
hash the counters were taken at."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_have_profiles():
    for key, t in bench.TRAFFIC.items():
        prof = os.path.join(ROOT, t["profile"])
        assert os.path.exists(prof), (key, t["profile"])
        text = open(prof, encoding="utf-8").read()
        assert t["sha"] in text, (key, "profile does not name the source hash of its counters")
        assert os.path.exists(os.path.join(bench.CSRC, t["src"])), key
        assert t["bytes"] > 0


def test_traffic_is_null_for_a_changed_source(monkeypatch):
    key = next(iter(bench.TRAFFIC))
    entry = dict(bench.TRAFFIC[key], sha="0" * 16)
    monkeypatch.setitem(bench.TRAFFIC, key, entry)
    assert bench.measured_traffic(key) is None
    assert bench.measured_traffic(("no-such-kernel",)) is None
