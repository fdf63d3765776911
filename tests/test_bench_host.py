"""Host-side pieces of bench.py (CPU; no GPU needed)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_traffic_record_was_taken_on_the_current_source():
    """roofline.traffic comes from the committed ncu record only while the
    z-sweep kernel's source hashes to the recorded value: the record in
    profiles/step_kernel_traffic.md must be retaken whenever that source changes."""
    b, note = bench.ncu_traffic("k_step_sweep", "f32", 1024 ** 3, 2)
    assert b is not None, "retake the DRAM traffic record: the z-sweep kernel's source changed"
    alg = 16 * 2 * 1024 ** 3
    assert 0.9 * alg <= b <= 1.1 * alg
    assert "scaled by 8" in note


def test_traffic_record_applies_only_to_its_precision_and_field_count():
    assert bench.ncu_traffic("k_step_sweep", "f32", 512 ** 3, 4) == (None, None)
    assert bench.ncu_traffic("k_step_sweep", "f64", 1024 ** 3, 2) == (None, None)
    assert bench.ncu_traffic("k_step_sweep", "f32", 512 ** 3, 2)[0] is not None


def test_fp64_pipe_roofline_only_for_the_measured_kernel_shape():
    r = bench.fp64_alu_roofline({"dims": 3, "nf": 2}, 16.0, "generic", 6793.1)
    assert r["bound"] == "alu" and abs(r["achieved"] - 16.0 * 32.2 / 1e3) < 1e-12
    assert abs(r["hbm_frac"] - 16.0 * 64 / 6793.1) < 1e-12
    assert bench.fp64_alu_roofline({"dims": 3, "nf": 4}, 8.0, "generic", 6793.1) is None
    assert bench.fp64_alu_roofline({"dims": 3, "nf": 2}, 14.0, "sweep", 6793.1) is None


def test_stats_error_is_relative_and_a_mean_against_the_spread():
    ref = {"mean": [1.0, 0.0], "var": [0.04, 1e-6], "E": 2.0, "a": 3.0, "ap": 0.5}
    got = {"mean": [1.001, 1e-4], "var": [0.0404, 1e-6], "E": 2.002, "a": 3.0, "ap": 0.5}
    e = bench.stats_error(got, ref)
    assert np.allclose(e["mean"], [1e-3, 1e-4 / 1e-3])
    assert np.allclose(e["var"], [1e-2, 0.0])
    assert abs(e["E"] - 1e-3) < 1e-12 and e["a"] == 0.0 and e["ap"] == 0.0
