"""Host logic of bench.py that needs no GPU: the clock summary taken during
the timed region, the gating of profiled DRAM traffic on the kernel's source
files, and the committed profile entries of the benchmark's kernels."""
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import bench as B
    return B


def test_clock_summary(bench):
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = bench.summarise_clocks(lines)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.summarise_clocks(["0, 1500, 2070, 1400, 0x8, Not Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.summarise_clocks([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_profiled_traffic_is_gated_on_the_kernels_sources(bench, tmp_path, monkeypatch):
    src = tmp_path / "k.cuh"
    src.write_text("kernel v1\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"files": ["k.cuh"], "source_hash": bench.files_hash(["k.cuh"]), "dram_bytes_per_symiter": 500.0}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k<16>": entry}))
    assert bench.profiled_traffic("k<16>", 2.0e6) == pytest.approx(1.0e9)
    assert bench.profiled_traffic("other<16>", 2.0e6) is None
    src.write_text("kernel v1 // a note\n/* and a block */\n")   # comments only: the code is the same
    assert bench.profiled_traffic("k<16>", 2.0e6) == pytest.approx(1.0e9)
    src.write_text("kernel v2\n")        # the kernel changed since the counters were taken
    assert bench.profiled_traffic("k<16>", 2.0e6) is None


def test_committed_profiles_cover_the_benchmark_kernels(bench):
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for name in bench.BENCH_KERNEL.values():
        assert name in t, name
    for name, ent in t.items():
        assert re.fullmatch(r"[0-9a-f]{16}", ent["source_hash"]), name
        # the counters were taken on the code the files hold now
        assert bench.files_hash(ent["files"]) == ent["source_hash"], f"{name}: profile is stale"
        assert ent["dram_bytes_per_symiter"] > 0
        for f in ent["files"]:
            assert os.path.exists(os.path.join(ROOT, f)), f
        assert os.path.exists(os.path.join(ROOT, ent["capture"])), ent["capture"]
        text = open(os.path.join(ROOT, ent["capture"])).read()
        assert "ncu" in text and "--clock-control none" in text


def test_error_rates_by_noise_level(bench):
    import numpy as np
    x = np.zeros((6, 4), np.int64)
    xh = x.copy()
    xh[1, 0] = 3          # level 1.5 dB: one symbol, two bits wrong
    xh[3, :] = 1          # level 1.0 dB: a whole frame, one bit per symbol
    r = bench.error_rates(xh, x, 4)
    assert r["1.0"] == {"fer": 0.5, "ser": 0.5, "ber": 4 / 16, "frames": 2}
    assert r["1.5"] == {"fer": 0.5, "ser": 1 / 8, "ber": 2 / 16, "frames": 2}
    assert r["2.0"]["fer"] == 0.0 and r["all"]["frames"] == 6


def test_fig1_statistic_on_a_hand_worked_example():
    """Fig. 1's statistic: P before the first iteration and after each one,
    frozen after a frame stops; gains dP over the iterations that ran,
    binned by the level they start from."""
    import numpy as np
    from bench_modes import fig1_gains, fig1_trajectory
    P0 = np.array([0.5, 0.25])
    P = np.array([[0.75, 1.0, 0.1],      # frame 0 stopped after 2 iterations (0.1: after the stop)
                  [0.25, 0.5, 0.75]])
    iters = np.array([2, 3])
    Pall = fig1_trajectory(P0, P, iters)
    np.testing.assert_array_equal(Pall, [[0.5, 0.75, 1.0, 1.0], [0.25, 0.25, 0.5, 0.75]])
    sums, cnts = fig1_gains(Pall, iters, np.array([0.0, 0.5, 1.0]))
    # bin [0, 0.5): frame 1's gains from 0.25 (0 and 0.25); bin [0.5, 1]:
    # frame 0's from 0.5 and 0.75, frame 1's from 0.5 (0.25 each)
    np.testing.assert_allclose(sums, [0.25, 0.75])
    np.testing.assert_array_equal(cnts, [2, 3])
