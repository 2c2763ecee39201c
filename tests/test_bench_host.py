"""Host logic of the benchmark (no GPU): the algorithmic bytes per cell it divides by, the
peak-pressure decay curve and its error statement, the clock-sample summary, and which ncu
counters it may attach to a measured kernel."""
import types

import numpy as np

import bench


def test_algorithmic_bytes_per_cell():
    # persistent state read once and written once: (f, rho) 2e, I 8 B, pmax e, v 2e
    assert bench.step_bytes_per_cell(8) == 96 and bench.step_bytes_per_cell(4) == 56
    kb8, kb4 = bench.kernel_bytes_per_cell(8), bench.kernel_bytes_per_cell(4)
    # a tile at rest moves as many bytes as the state: (f, rho), I and (p, c^2) read and
    # written, its vertex written
    assert kb8["k_rest_tiles"] == 96 and kb4["k_rest_tiles"] == 56
    assert kb8["k_step_fused"] == 96 and kb4["k_step_fused"] == 56
    # the copy beside the tile kernel moves the same tiles
    assert all(kb8[k] == 96 for k in bench.REST_KERNELS)


def test_peak_decay_bins_by_distance_from_the_impact_point():
    rc = np.array([0.5, 1.5, 2.5])
    zc = np.array([0.5, 1.5])
    z_surface = 2.0
    pmax = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    # distances: row z=0.5 -> hypot(rc, 1.5); row z=1.5 -> hypot(rc, 0.5)
    curve = bench.peak_decay(pmax, rc, zc, z_surface, 1.0, 4)
    d = np.hypot(rc[None, :], zc[:, None] - z_surface)
    ref = np.zeros(4)
    for (j, i), v in np.ndenumerate(pmax):
        k = min(int(d[j, i]), 4)
        if k < 4:
            ref[k] = max(ref[k], v)
    assert np.array_equal(curve, ref)


def test_decay_errors_over_the_bins_above_the_floor():
    p64 = np.array([100.0, 50.0, 10.0, 0.5])
    p32 = np.array([101.0, 49.0, 10.0, 0.9])
    e = bench.decay_errors(p32, p64, floor=0.01)
    assert e["bins"] == 3                       # 0.5 is below 1 % of 100
    assert abs(e["max"] - 0.02) < 1e-12 and abs(e["mean"] - 0.01) < 1e-12


def test_clock_summary_reads_the_samples_and_the_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070 MHz, 2070 MHz, 600.0 W, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 2000, 2070, 650.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 1500, 2070, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = bench.ClockSampler(0)
    s.path = str(path)
    out = s.summary()
    # the two samples above 200 W are the loaded ones (the unit suffixes do not parse)
    assert out["samples"] == 2 and out["reasons"] == ["sw_power_cap"]
    assert out["sm_mhz"] == 2000.0 and out["sm_max_mhz"] == 2070.0


def test_ncu_counters_only_for_the_workload_they_were_taken_on():
    args = types.SimpleNamespace(workload="large_4000", steps=20, warmup=5)
    tr, kind = bench._traffic("k_rest_tiles", "fp64", args)
    assert tr is not None and "same 20 launches" in kind
    args2 = types.SimpleNamespace(workload="large_4000", steps=2000, warmup=5)
    assert bench._traffic("k_rest_tiles", "fp64", args2)[0] is None
    saved = dict(bench._COUNTERS_STALE)
    try:
        bench._COUNTERS_STALE["fp64"] = {"k_rest_tiles"}
        assert bench._traffic("k_rest_tiles", "fp64", args) == (None, "counters stale")
    finally:
        bench._COUNTERS_STALE.clear()
        bench._COUNTERS_STALE.update(saved)


def test_tile_kernel_traffic_withheld_beside_the_copy_kernel():
    """With the tiles at rest copied beside the tile kernel, the FP64 tile kernel is another
    instantiation sharing its SMs with the copies: the DRAM traffic of the capture is not
    reported for it, its FP64 operation count (same arithmetic) is."""
    args = types.SimpleNamespace(workload="large_4000", steps=20, warmup=5)
    assert bench._traffic("k_step_fused", "fp64", args)[0] is not None
    assert bench._traffic("k_step_fused", "fp64", args, beside=True)[0] is None
    assert bench._FUSED_FULL_SIZE["fp64"]["k_step_fused"]["flops"] > 0
    assert bench._traffic("k_rest_copy", "fp64", args)[0] is None
