"""Host-side arithmetic of the benchmark line (CPU): the HBM-roofline fraction
of a zone-update rate and the mixed form's FP32-pipe figures."""
import json
import os

import pytest

import bench


def test_hbm_fraction_counts_the_fp64_state_read_and_written_once():
    peak, src = bench.hbm_peak_gbs()
    assert peak > 0 and src
    h = bench.hbm_fraction(1e9)
    assert h["bytes_per_zone_update"] == 80
    assert h["achieved_gbs"] == pytest.approx(80.0)
    assert h["frac"] == pytest.approx(80.0 / peak)


def test_hbm_peak_is_the_measured_copy_bandwidth_when_recorded():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        assert bench.hbm_peak_gbs()[0] == 6800.0
        return
    with open(path) as f:
        assert bench.hbm_peak_gbs()[0] == float(json.load(f)["hbm_gbs"])


def test_fp32_pipe_counts_the_fp32_stages_over_the_step_and_their_own_time():
    n = (256, 256, 256)
    flops = sum(bench.FLOPS_PER_UNIT[s] * bench.units_per_launch(s, n) for s in bench.FP32_STAGES_MIXED)
    stage_ms = {"prim": 1.10, "flatten": 0.15, "slopes": 0.002, "trace": 1.44, "riemann": 0.002,
                "ctu1": 1.71, "ctu2": 1.07, "update": 1.16}
    f = bench.fp32_pipe(n, 6.71, stage_ms)
    own_ms = 0.15 + 0.002 + 1.44 + 0.002 + 1.71 + 1.07
    assert f["algorithmic_tflops_whole_step"] == pytest.approx(flops / 6.71e-3 / 1e12)
    assert f["algorithmic_tflops_in_fp32_stages"] == pytest.approx(flops / (own_ms * 1e-3) / 1e12)
    assert f["frac_whole_step"] == pytest.approx(f["algorithmic_tflops_whole_step"] / f["peak_tflops"])
    assert 0 < f["frac_whole_step"] < f["frac_in_fp32_stages"] < 1
    assert bench.fp32_pipe(n, 6.71, {})["frac_in_fp32_stages"] is None
