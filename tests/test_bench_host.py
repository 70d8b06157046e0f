"""Host logic of bench.py that needs no GPU: the DRAM traffic taken from an ncu summary only while the kernel's
sources hash to the captured ones, the clock-record parsing that rejects throttled runs, and the single-rank
reductions."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_profiled_traffic_follows_the_kernel_sources(tmp_path):
    """A summary whose source hash is the kernel's current one gives its DRAM bytes; any other hash gives None (the
    counters were taken on another kernel), and so does a missing summary."""
    os.makedirs(tmp_path / "profiles")
    name = "match_tc_kernel_some_workload"
    cur = bench._kernel_source_hash("gm_match_tc.cu")
    for sha, want in ((cur, 5.5e8), ("0" * 64, None)):
        with open(tmp_path / "profiles" / f"{name}.txt", "w") as fh:
            fh.write(f"kernel: match_tc_kernel\nsource_sha256: {sha}\ndram_bytes_per_launch: 5.5e8\n")
        assert bench._profiled_traffic("match_tc_kernel", "gm_match_tc.cu", "some_workload", root=str(tmp_path)) == want
    assert bench._profiled_traffic("match_tc_kernel", "gm_match_tc.cu", "absent", root=str(tmp_path)) is None


def test_profiles_name_their_commands():
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        with open(os.path.join(ROOT, "profiles", name)) as fh:
            text = fh.read()
        assert "ncu " in text and "bench.py" in text, name


def test_clock_summary_flags_throttling(tmp_path):
    rows = ["0, 2070, 2070, 180.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 420.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1500, 2070, 600.0, 0x8, Active, Not Active, Not Active, Active"]
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 1980.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"] and s["power_w_max"] == 600.0
    c.path = str(tmp_path / "missing.csv")
    assert bench.ClockSampler.summary(c)["reasons"] == ["unsampled"]


def test_single_rank_reductions():
    assert bench._reduce(3.25, "max", 1, "cpu") == 3.25
    assert bench._reduce(1200, "sum", 1, "cpu") == 1200.0
    import scenes
    assert bench._facade_seed(0) == scenes.SEED_BASE + 2
