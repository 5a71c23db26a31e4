"""Host-side logic of the benchmark (no GPU): the operation count behind the
roofline, the guard that reports the profiled DRAM traffic only for the
kernel sources it was measured on, the clock record parsed from nvidia-smi
samples, and the per-rank sharding of the step counters."""
import os
import tempfile

import bench


def test_operation_count_is_the_stage_table():
    assert bench.OPS_PER_BUNCH == sum(bench.OPS_PER_BUNCH_FP32.values()) == 215
    assert bench.OPS_PER_STEP == sum(bench.OPS_PER_STEP_FP32.values()) == 113
    # Philox per bunch: 8 full rounds plus the bunch index's share of the
    # first two (the key schedule is per launch, the step's share per step)
    assert bench.OPS_PER_BUNCH_FP32["philox4x32_10"] == 8 * 8 + 3 + 4
    assert bench.OPS_PER_STEP_FP32["philox_step_share"] == 2 * (2 + 2)
    assert bench.FP64_OPS_PER_BUNCH == 215 - bench.OPS_PER_BUNCH_FP32["philox4x32_10"]


def test_rooflines_from_the_counts():
    r = bench.alu_roofline(6.4e7, 2e6, 0.8, 152, 2070.0)
    ops = 215 * 6.4e7 + 113 * 2e6
    assert abs(r["achieved"] - ops / 0.8e-3 / 1e12) < 1e-9
    assert abs(r["peak"] - 152 * 128 * 2.07e9 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["peak_source"].startswith("derived")
    f = bench.fp64_roofline(6.4e7, 2e6, 18.0, 152, 2070.0)
    assert abs(f["frac"] - (144 * 6.4e7 + 64 * 2e6) / 18e-3 / (152 * 2 * 2.07e9)) < 1e-12


def test_traffic_only_for_the_profiled_sources(monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_PER_STEP", {"vertical_1tev": (76.5, "ab" * 8)})
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "ab" * 8)
    assert bench._traffic("vertical_1tev", 2_000_000) == 153_000_000   # scaled by steps
    assert bench._traffic("inclined_20tev", 1) is None                 # not profiled
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "0" * 16)        # sources changed
    assert bench._traffic("vertical_1tev", 2_000_000) is None


def test_kernel_hash_covers_the_kernel_sources():
    h = bench._kernel_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    for f in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2006_14927_gb300", "csrc", f))


def test_clock_record_from_samples():
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1010.4, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 990.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = path
    rec = cs.summary()
    os.unlink(path)
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert rec["samples"] == 3


def test_clock_record_without_samples():
    cs = bench.ClockSampler(0)
    cs.path = os.path.join(tempfile.gettempdir(), "no-such-clock-file.csv")
    assert cs.summary()["reasons"] == ["unsampled"]


def test_ranks_get_disjoint_step_counters():
    n = 2_000_000
    bases = [bench.shard(r, n, 2)[1] for r in range(8)]
    seeds = [bench.shard(r, n, 2)[0] for r in range(8)]
    assert bases == [r * n for r in range(8)]
    assert len(set(seeds)) == 8
