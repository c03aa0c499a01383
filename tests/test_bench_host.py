"""Host-side arithmetic of the benchmark line (CPU): the HBM-roofline fraction
of a zone-update rate."""
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
