"""Host-side logic of bench.py (no GPU): the roofline arithmetic of the
dominant kernel and the parsing of the clock samples taken during the timed
region."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_roofline_takes_the_kernel_with_the_most_time():
    n = 16384
    kms = {0: 947.0, 1: 1443.0}        # total ms over the timed region
    kcnt = {0: 1000, 1: 1000}
    kinds = {0: "x_band_kernel", 1: "y_coop_kernel"}
    alg = {0: 12 * n * n, 1: 20 * n * n}
    r = bench._roofline(kms, kcnt, kinds, alg, "ricker_16384")
    assert r["kernel"] == "y_coop_kernel" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["avg_launch_ms"] == pytest.approx(1.443)
    assert r["achieved"] == pytest.approx(20 * n * n / 1.443e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == bench.NCU_TRAFFIC[("ricker_16384", "y_coop_kernel")]
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")  # written per machine, not versioned
    if os.path.exists(peaks):
        with open(peaks) as f:
            assert r["peak"] == float(json.load(f)["hbm_gbs"]) and r["peak_source"] == "measured"
    else:
        assert r["peak"] == 6800.0 and r["peak_source"] == "fallback"
    # another workload has no captured traffic
    assert bench._roofline(kms, kcnt, kinds, alg, "ricker_4096")["traffic"] is None
    # the x sweep dominates when it takes longer
    r2 = bench._roofline({0: 2000.0, 1: 1000.0}, kcnt, kinds, alg)
    assert r2["kernel"] == "x_band_kernel"
    assert r2["achieved"] == pytest.approx(12 * n * n / 2.0e-3 / 1e9)


def test_clock_samples_median_and_reasons():
    lines = [
        "2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1320.4, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1300.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "garbage",                                                                 # skipped
    ]
    c = bench.ClockSampler.parse(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    hot = bench.ClockSampler.parse(
        ["1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.ClockSampler.parse([]) is None


def test_gpus_two_starts_two_ranks_that_agree():
    """`bench.py --gpus 2` outside torchrun starts two ranks itself (on
    127.0.0.1); each sees WORLD_SIZE 2 and its own RANK."""
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2",
                        "--print-ranks"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert sorted(d["rank"] for d in lines) == [0, 1]
    assert all(d["world_size"] == 2 for d in lines)
    assert sorted(d["local_rank"] for d in lines) == [0, 1]


def test_custom_workload_needs_a_shape():
    with pytest.raises(SystemExit):
        bench.parse_args(["--workload", "custom"])
    a = bench.parse_args(["--workload", "custom", "--nx", "64", "--ny", "32", "--time-steps", "3"])
    p = bench.make_problem(bench.WORKLOADS["custom"], a)
    assert (p.nx, p.ny, p.time_steps) == (64, 32, 3)
    assert p.m.shape == (32, 64) and p.wavelet.shape == (5,)
    assert p.tau == pytest.approx(0.5 / 65 / float(p.m.max()) ** 0.5)
