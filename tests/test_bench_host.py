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


def test_peak_fractions_of_matvec_and_solve():
    """The matvec's work is the three FMM passes' kernel_work; the solve's adds E y to each
    of its applications; rates against the roofline's peak."""
    counts = {"N": 1000, "p2p_pairs": 50000, "m2m": 100, "m2l": 2000, "l2l": 100,
              "w_pairs": 300, "x_pairs": 300}
    bcounts = {"p2l_pairs": 400, "direct_pairs": 50, "global_centres": 0, "terms": 32}
    line = {"solve": {"counts": counts, "border_counts": bcounts, "tree": {"p": 9},
                      "fp64_applies": 7, "solve_ms": 20.0},
            "roofline": {"unit": "TFLOP/s", "peak": 1.25, "peak_source": "nominal"},
            "matvec": {"fp64": {"ms": 2.0}}}
    Q, N = 10, 1000
    up = 8 * Q * N + (2 * Q * (Q + 1) + 14 * Q) * 100
    down = (4 * Q * Q + 14 * Q) * 2000 + (2 * Q * (Q + 1) + 14 * Q) * 100 + 8 * Q * 300
    leaf = 11 * 50000 + 8 * Q * N + 8 * Q * 300 + 10 * N
    esum = 8 * 32 * 400 + (2 * 32 * 33 + 14 * 32) * 100 + 8 * 32 * N + 8 * 50 + 10 * N
    pf = bench.peak_fractions(line)
    assert abs(pf["matvec"]["gflop"] - (up + down + leaf) / 1e9) < 1e-15
    assert abs(pf["matvec"]["achieved"] - (up + down + leaf) / 2e-3 / 1e12) < 1e-15
    assert abs(pf["solve"]["gflop"] - 7 * (up + down + leaf + esum) / 1e9) < 1e-15
    assert abs(pf["solve"]["frac"] - 7 * (up + down + leaf + esum) / 20e-3 / 1e12 / 1.25) < 1e-15
    assert bench.peak_fractions({"solve": {}}) is None
    line["matvec"] = None
    assert bench.peak_fractions(line) is None
