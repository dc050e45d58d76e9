"""Host logic of bench.py on CPU: the roofline block's arithmetic and source selection, and the parser of the
clock samples taken during the timed region (the rejection rules read its reasons)."""
import os

import pytest

import bench


def _counts(sweep0=0, taps0=0, plane=0, taps_plane=0, ransac=0, init=0):
    from paper_1804_03787_gb300 import gpm
    c = [0] * gpm.COUNTERS
    c[gpm.COUNT_SWEEP0], c[gpm.COUNT_SWEEP0_TAPS] = sweep0, taps0
    c[gpm.COUNT_SWEEP_PLANE], c[gpm.COUNT_SWEEP_PLANE_TAPS] = plane, taps_plane
    c[gpm.COUNT_RANSAC], c[gpm.COUNT_INIT] = ransac, init
    return c


def test_roofline_block_takes_the_top_class_and_divides_by_its_launch_time():
    # 1e9 square-patch evaluations summing 5e10 taps at 6 FP32 operations each, over 160 launches taking 100 ms in
    # all; the initial field's evaluations are not the sweep's work
    prof = {"pm_sweep": (100.0, 160), "ransac": (50.0, 40), "pm_sweep_plane": (30.0, 64)}
    evals = _counts(sweep0=1e9, taps0=5e10, init=7e8)
    blk = bench.roofline_block(prof, evals, 152, {"sm_mhz": 2000.0}, {"hbm_gbs": 6783.0}, steps=10)
    assert blk["kernel"] == "pm_sweep" and blk["bound"] == "alu"
    assert blk["share"] == pytest.approx(100 / 180)
    assert blk["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e12)                  # nominal: no probe given
    assert "nominal" in blk["peak_source"]
    assert blk["achieved"] == pytest.approx(5e10 / 160 * 6 / (100 / 160 * 1e-3) / 1e12)
    assert blk["frac"] == pytest.approx(blk["achieved"] / blk["peak"])
    assert blk["per_launch"]["taps_per_evaluation"] == pytest.approx(50.0)
    assert blk["avg_launch_ms"] == pytest.approx(100 / 160)
    assert "profiled replay" in blk["avg_launch_source"]
    hv = blk["hbm_view"]                                                            # 48 B per visit, W*H visits
    assert hv["algorithmic_bytes_per_launch"] == 1024 * 436 * 48
    assert hv["achieved_gbs"] == pytest.approx(1024 * 436 * 48 / (100 / 160 * 1e-3) / 1e9)
    assert hv["frac"] == pytest.approx(hv["achieved_gbs"] / 6783.0)
    assert blk["traffic"] == bench.TRAFFIC_PER_LAUNCH["pm_sweep"][0]                # ncu capture of this kernel
    assert blk["traffic_source"].startswith("profiles/") and blk["issue_view"]["issue_slots_busy"] > 0


def test_roofline_block_takes_a_single_kernel_over_the_ransac_class():
    """The RANSAC class holds three kernels (fit, refit solve, finish): with the largest class share it still
    yields to the largest single-kernel class."""
    prof = {"pm_sweep": (100.0, 160), "ransac": (140.0, 240), "pm_sweep_plane": (90.0, 640)}
    blk = bench.roofline_block(prof, _counts(sweep0=1e9, taps0=5e10), 152, {"sm_mhz": 2000.0}, {}, steps=10)
    assert blk["kernel"] == "pm_sweep" and blk["share"] == pytest.approx(100 / 330)


def test_roofline_block_prefers_the_timed_region_and_the_measured_peak():
    prof = {"pm_sweep": (100.0, 160)}
    fp32 = {"lane_ops_per_clk": 19000.0}
    blk = bench.roofline_block(prof, _counts(sweep0=1e9, taps0=8.1e10), 152, {"sm_mhz": None},
                               {"sm_max_mhz": 2070.0}, steps=10, timed={"pm_sweep": (80.0, 160)}, fp32=fp32)
    assert blk["avg_launch_ms"] == pytest.approx(0.5) and "timed region" in blk["avg_launch_source"]
    assert blk["achieved"] == pytest.approx(8.1e10 / 160 * 6 / 0.5e-3 / 1e12)
    assert blk["peak"] == pytest.approx(19000.0 * 2070e6 / 1e12)                   # measured rate, max clock
    assert "measured" in blk["peak_source"]
    other = bench.roofline_block({"fill": (5.0, 8)}, _counts(), 152, {"sm_mhz": 2000.0}, {}, steps=1)
    assert other["achieved"] is None and other["frac"] is None and other["traffic"] is None


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_median_and_throttle_reasons(tmp_path):
    c = bench.Clocks("0")
    c.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",     # unreadable: skipped
            "garbage"]
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    c.proc, c.f = _FakeProc(), open(os.devnull, "w")
    got = c.stop()
    assert got["sm_mhz"] == 2055 and got["sm_max_mhz"] == 2070 and got["samples"] == 3
    assert got["reasons"] == ["sw_power_cap"]
    rows[0] = "0, 1500, 2070, 900.1, 0x0, Active, Not Active, Not Active, Not Active"
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    c.f = open(os.devnull, "w")
    assert c.stop()["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi_says_so():
    c = bench.Clocks("0")
    c.proc = None
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the oracle on the host and prints one JSON line with the contract's
    keys, its own value repeated as the CPU baseline and as the end-to-end figure (no device copies)."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=bench.ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "pairs/s" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    # ms_per_step is the measured time of a step's sample (a crop); value counts the crop as its fraction of a pair
    frac = d["config"]["pairs_per_step"]
    assert 0.1 < frac < 0.2
    assert abs(d["ms_per_step"] - 1e3 * frac / d["value"]) < 1e-6 * d["ms_per_step"]
