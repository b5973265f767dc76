"""Host logic of bench.py that needs no GPU: the clock record read from
nvidia-smi, the rule that rejects a timed region, the whole-job replica value
and the algorithmic flop count behind the roofline."""
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _summary(lines):
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    clk = bench.ClockSampler()
    clk.path = path
    out = clk.summary()
    assert not os.path.exists(path)          # the record is removed once read
    return out


def test_clock_record_median_max_and_reasons():
    quiet = "Not Active, Not Active, Not Active, Not Active"
    out = _summary([
        "2070, 2070, 350.1, 0x0000000000000000, " + quiet,
        "1980, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 420.0, 0x0000000000000000, " + quiet,
        "garbage line",
        "[N/A], 2070, 1.0, 0x0, " + quiet,
    ])
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}


def test_empty_clock_record():
    assert _summary([]) is None


def test_rejection_rule():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(None)
    assert not bench.clocks_rejected(dict(ok, reasons=["sw_power_cap"], sm_mhz=1440.0))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1500.0))          # held low, no reason
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1900.0))


def test_replica_value_is_whole_job_throughput():
    # 4 steps of 1000 units on each of 2 ranks, the slowest rank took 2 s
    assert bench.replica_value(1000.0, 4, 2.0, 2) == 4000.0


def test_algorithmic_flops_of_the_bench_workload():
    # 24 m n + 12 N m + 40 m + 4 n^2 + 4 n n_eq at m = 100, n = 11, N = 12, n_eq = 3
    assert bench.algorithmic_flops_per_sample_iter(100, 11, 12) == 26400 + 14400 + 4000 + 484 + 132


def test_traffic_is_reported_only_for_the_captured_kernel_source(monkeypatch):
    """The DRAM traffic of the roofline comes from an ncu capture; it is
    reported only while the fused kernel's source still has the hash recorded
    with the capture, and is null otherwise."""
    import bench
    sha = bench.fused_source_sha256()
    monkeypatch.setattr(bench, "FUSED_TRAFFIC", {"source_sha256": sha, "capture": "cap",
                                                 "bytes": {(1, 8): 12345}})
    assert bench.fused_traffic((1, 8)) == (12345, "cap")
    assert bench.fused_traffic((1, 4))[0] is None
    monkeypatch.setattr(bench, "FUSED_TRAFFIC", {"source_sha256": "0" * 64, "capture": "cap",
                                                 "bytes": {(1, 8): 12345}})
    assert bench.fused_traffic((1, 8))[0] is None
