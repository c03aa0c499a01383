"""The allocation-free time-step entry point (hydro_compute_dt_noalloc).

Callers that cannot allocate device memory when they need a time step (a
process whose device memory all belongs to its own pool, or a loop that cannot
afford cudaMalloc/cudaFree) use this call instead of hydro_compute_dt, which
needs a handle with caller-allocated scratch.  It must give the same per-box
time steps.  Two calls in a row on different box sets check that the shared
static scratch is fully rewritten and cleared by each call.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2007_05218_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu


def _dt_both_ways(problems):
    import torch
    B = hydro.Boxes(problems)
    ref = B.compute_dt().clone()          # existing entry point, through the handle
    out = torch.full((B.nboxes,), -1.0, dtype=torch.float64, device="cuda")
    hydro.hydro_compute_dt_noalloc(B.descs, B.state, out)
    torch.cuda.synchronize()
    got, want = out.cpu().numpy(), ref.cpu().numpy()
    B.close()
    return got, want


def test_noalloc_dt_matches_handle_dt_on_two_calls_in_a_row():
    fast = [inputs.sedov((17, 16, 18), seed=2), inputs.density_wave((20, 12, 9), seed=3),
            inputs.kelvin_helmholtz((12, 16, 10), seed=4)]
    slow = [inputs.uniform((8, 9, 10), vel=(0.01, 0.0, 0.0), p=1e-3, bc="outflow"),
            inputs.uniform((6, 5, 7), vel=(0.0, 0.02, 0.0), p=2e-3, bc="periodic")]
    for problems in (fast, slow):  # the second call has fewer boxes and far smaller speeds
        got, want = _dt_both_ways(problems)
        np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)


def test_noalloc_dt_rejects_more_boxes_than_its_scratch_holds():
    import torch
    d = hydro.desc_of(inputs.uniform(4))
    descs = [d] * 1025
    dt = torch.zeros(1025, dtype=torch.float64, device="cuda")
    state = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(hydro.HydroError) as e:
        hydro.hydro_compute_dt_noalloc(descs, state, dt)
    assert e.value.code == hydro.HYDRO_ERR_INVALID
    assert "1024" in str(e.value)
