"""bench.py's accounting, checked on the CPU: the roofline's algorithmic bytes per node
(one pass reads the moduli, u and f once and writes once; a full red-black sweep of FP32
general moduli is 120 B/node over two half-sweep launches), the bytes the colour-split
kernels are designed to move, the FP64 flop count of a residual row, the peak taken from
the measured-peaks file (or the stated fallback), and the parsing of the clock samples
that decides whether a run is kept."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_per_node():
    # FP32, 21 moduli: (84 moduli + 12 u + 12 f + 12 written) / 2 half-sweeps
    assert bench.alg_bytes_per_node("sweep32", 21) == 60
    assert 2 * bench.alg_bytes_per_node("sweep32", 21) == 120
    assert bench.alg_bytes_per_node("sweep32", 2) == (8 + 36) / 2
    assert bench.alg_bytes_per_node("sweep64", 21) == (168 + 72) / 2
    # the refinement residual: FP64 moduli, u, f read, r written as FP32
    assert bench.alg_bytes_per_node("resid64_mixed", 21) == 168 + 24 + 24 + 12
    assert bench.alg_bytes_per_node("resid32", 21) == 84 + 36


def test_issued_bytes_of_the_colour_split_half_sweep():
    # 39 floats per active node (half the nodes), u and f lines, every output row written
    assert bench.issued_bytes_per_node("sweep32", 21) == 39 * 4 / 2 + 36 == 114
    assert bench.issued_bytes_per_node("sweep32", 2) == 8 + 36
    assert bench.flops_per_node_resid64(21) == 249 and bench.flops_per_node_resid64(2) == 161


def test_hbm_peak_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6787.2, "bf16_tflops": 1931.3}))
    assert bench.measured_peaks() == (6787.2, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("not json")
    assert bench.measured_peaks() == (bench.FALLBACK_HBM_GBS, "fallback")


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks_from(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(l + "\n" for l in lines))
    c = bench.Clocks(0)
    c.proc, c.path = _Done(), str(path)
    return c.stop()


def test_clock_samples_median_and_throttle_reasons(tmp_path):
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    ok = "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1900, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1390.0, 0x0000000000000040, Active, Active, Not Active, Not Active"
    out = _clocks_from(tmp_path, [ok, ok, capped, "garbage line", "0, [N/A], 2070, 1.0, 0x0, a, b, c, d"])
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    out = _clocks_from(tmp_path, [ok, hot, hot])
    assert out["sm_mhz"] == 1500 and out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert _clocks_from(tmp_path, ["garbage"]) is None
    assert bench.Clocks(0).stop() is None          # never started: no record


def test_rve_oracle_timing_reports_one_core_and_all_core_rates():
    """The CPU baseline's timed oracle solves of a periodic RVE (spawned single-threaded
    workers): one solve on one core, one per worker at once, each converged to 1e-8."""
    out = bench.rve_oracle_timed(2, n=9)
    assert out["cycles"] > 0 and out["rel_residual"] <= 1e-8
    one, many = out["one_core"], out["all_cores"]
    assert one["seconds_per_solve"] > 0 and one["solves_per_s"] == 1.0 / one["seconds_per_solve"]
    assert many["cores"] == many["solves"] == 2 and many["solves_per_s"] == 2 / many["wall_s"]
    assert many["mean_seconds_per_solve"] > 0
