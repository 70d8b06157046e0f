"""Host logic of bench.py that needs no GPU: the committed ncu summary of the dominant kernel still matches the
kernel's sources (so the bench reports its DRAM traffic), the clock-record parsing that rejects throttled runs, and
the single-rank reductions."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_dominant_kernel_profile_matches_sources():
    traffic = bench._profiled_traffic("match_tc_kernel", "gm_match_tc.cu", bench.WORKLOAD)
    assert traffic is not None and traffic > 1e8


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
