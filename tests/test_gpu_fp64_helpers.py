"""The device arithmetic helpers the FP64 kernels rest on, checked on the GPU
(needs a GB300 and nvcc): bit-pattern sign tests, comparisons, min/max,
exact halving, the |x| > 2|y| test, the integer-pipe FP64 -> FP32 rounding and
the integer-pipe FP64 product against IEEE operations bit for bit over every
exponent; Newton-refined reciprocal and square root within 2 ulp and
reciprocal square root within 2^-51.5 relative over normal arguments.
"""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2007_05218_gb300", "csrc")


def test_fp64_helpers_match_ieee(tmp_path):
    from paper_2007_05218_gb300 import build
    exe = str(tmp_path / "fp64_helpers_check")
    cmd = [build.nvcc(), "-O3", "-std=c++17", *build.ARCH, "-I", CSRC, "-o", exe,
           os.path.join(HERE, "fp64_helpers_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0 and "PASS" in r.stdout, r.stdout + r.stderr
