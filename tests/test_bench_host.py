"""Host logic of the bench's roofline (CPU): the DRAM traffic per launch comes from the
ncu captures in profiles/traffic.json only while they match the FMM sources they were taken
on (a kernel changed since the capture reports null traffic)."""
import json
import os

import bench

KEYS = (("down", 22, 32), ("leaf", 22, 32), ("up", 22, 32), ("down", 22, 48), ("leaf", 22, 48),
        ("up", 22, 48), ("down32", 12, 48), ("leaf32", 12, 48), ("up32", 12, 48))


def test_traffic_follows_the_captures_of_the_current_sources():
    tj = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    current = tj["src_hash"] == bench.src_hash()
    for kernel, p, leaf in KEYS:
        b = bench.traffic_for(kernel, p, leaf)
        if current:  # the passes of the autotuned settings and the float defaults
            assert isinstance(b, int) and b > 0
        else:
            assert b is None
    assert bench.traffic_for("down", 23, 32) is None  # no capture at that order


def test_traffic_is_dropped_when_the_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "src_hash", lambda: "0" * 16)
    for kernel, p, leaf in KEYS:
        assert bench.traffic_for(kernel, p, leaf) is None
