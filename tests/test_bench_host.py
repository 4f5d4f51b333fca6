"""Host-side helpers of bench.py that decide whether a run is valid (no GPU):
the clock record taken during the timed region, and the CPU-baseline line."""
import os
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _FakeSampler:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _record(lines):
    f = tempfile.NamedTemporaryFile("w", suffix=".csv", delete=False)
    f.write("\n".join(lines) + "\n")
    f.close()
    return f.name


def test_clock_record_median_max_and_reasons():
    import bench
    # index, clocks.sm, clocks.max.sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    path = _record([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, 900, 2070, 300.0, 0x8, Active, Not Active, Not Active, Not Active",   # another GPU
        "garbage line",
    ])
    c = bench.clocks_stop(_FakeSampler(), path, 0)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]          # kept and noted; GPU 1's slowdown ignored
    assert not os.path.exists(path)


def test_clock_record_flags_hardware_slowdown():
    import bench
    path = _record([
        "2, 1500, 2070, 800.0, 0x8, Active, Active, Not Active, Not Active",
        "2, 1490, 2070, 800.0, 0x8, Active, Not Active, Not Active, Not Active",
    ])
    c = bench.clocks_stop(_FakeSampler(), path, 2)
    assert set(c["reasons"]) == {"hw_slowdown", "hw_thermal_slowdown"}
    assert c["sm_mhz"] == pytest.approx(1495.0)


def test_clock_record_without_sampler():
    import bench
    c = bench.clocks_stop(None, None, 0)
    assert c["sm_mhz"] is None and c["reasons"]


def test_cpu_baseline_line(monkeypatch):
    """The CPU baseline line is the oracle TE-FMM sample's throughput with the
    cores it used (CPU time over wall time)."""
    import bench
    monkeypatch.setattr(bench, "oracle_fmm_sample", lambda w, n, warm=True: (20.0, 1.5, "sample", n * 2000))
    cb = bench.cpu_baseline(None, n_targets=2)
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT
    assert cb["value"] == pytest.approx(2 * 2000 / 20.0)
    assert cb["cores"] == 1.5 and cb["sample"] == "sample"


def test_stored_direct_sum_reference():
    """The stored 1000-target direct sum of the 2M workload: default_rng(1)'s
    sample of the 2M points, finite non-zero values, read in order."""
    import numpy as np
    import bench

    class Wk:
        name = "three_layer_slabs_n2M_p10"
        src = np.zeros((2_000_000, 3))
    idx, ref, where = bench.reference_at(Wk, 1000)
    assert where.startswith("tests")
    assert np.array_equal(idx, np.random.default_rng(1).choice(2_000_000, 1000, replace=False))
    assert np.all(np.isfinite(ref)) and np.all(np.abs(ref) > 0)
    idx2, ref2, _ = bench.reference_at(Wk, 100)
    assert np.array_equal(idx2, idx[:100]) and np.array_equal(ref2, ref[:100])


def test_err_stats_follow_the_papers_measures():
    """Err_2 and Err_max (Sec. 5), overall and per layer, on a hand-made case."""
    import numpy as np
    import bench
    ref = np.array([1.0, 2.0j, -2.0, 4.0])
    phi = ref + np.array([0.1, 0.0, 0.2j, 0.0])
    s = bench.err_stats(phi, ref, [0, 0, 1, 1])
    assert s["rel_l2"] == pytest.approx(np.sqrt((0.01 + 0.04) / (1 + 4 + 4 + 16)))
    assert s["max_rel"] == pytest.approx(0.1)              # 0.1 / 1 beats 0.2 / 2
    assert s["per_layer"]["0"]["rel_l2"] == pytest.approx(np.sqrt(0.01 / 5))
    assert s["per_layer"]["1"]["max_rel"] == pytest.approx(0.1)
    assert s["per_layer"]["1"]["rel_l2"] == pytest.approx(np.sqrt(0.04 / 20))
