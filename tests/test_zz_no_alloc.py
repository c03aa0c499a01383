"""The allocation-free time-step entry point (hydro_compute_dt_noalloc).

Callers that cannot allocate device memory when they need a time step (a
process whose device memory all belongs to its own pool, or a loop that cannot
afford cudaMalloc/cudaFree) use this call instead of hydro_compute_dt, which
needs a handle with caller-allocated scratch.  It forms the signal speeds with
the same device code as a handle, so under the default limiter it must give the
same per-box time steps bit for bit.  Two calls in a row on different box sets
check that the shared static scratch is fully rewritten and cleared by each
call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2007_05218_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu


def _dt_both_ways(descs, problems, stream=None):
    import torch
    B = hydro.Boxes(descs)
    for k, p in enumerate(problems):
        B.set_interior(k, p.U)
    torch.cuda.synchronize()
    ref = torch.full((B.nboxes,), -2.0, dtype=torch.float64, device="cuda")
    out = torch.full((B.nboxes,), -1.0, dtype=torch.float64, device="cuda")
    hydro.hydro_compute_dt(B.h, ref, stream)   # existing entry point, through the handle
    hydro.hydro_compute_dt_noalloc(B.descs, B.state, out, stream)
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
        got, want = _dt_both_ways([hydro.desc_of(p) for p in problems], problems)
        assert np.all(want > 0)
        np.testing.assert_array_equal(got, want)


def test_noalloc_dt_full_box_table_with_mixed_boxes_on_a_side_stream():
    """Exactly HYDRO_NOALLOC_MAX_BOXES boxes (uneven, some mixed precision,
    perturbed states) on a non-default stream, twice in a row."""
    import torch
    rng = np.random.default_rng(11)
    for rep in range(2):
        probs, descs = [], []
        for k in range(1024):
            n = tuple(int(x) for x in rng.integers(4, 10, size=3))
            pr = inputs.uniform(n, rho=float(rng.uniform(0.5, 2.0)), vel=tuple(rng.uniform(-1.0, 1.0, 3)),
                                p=float(rng.uniform(0.05, 3.0)), bc="outflow")
            pr.U[0] *= 1.0 + 0.05 * rng.uniform(-1.0, 1.0, pr.U[0].shape)
            pr.U[4] *= 1.0 + 0.05 * rng.uniform(-1.0, 1.0, pr.U[4].shape)
            probs.append(pr)
            descs.append(hydro.desc_of(pr, hydro.HYDRO_MIXED if (k + rep) % 5 == 0 else hydro.HYDRO_FP64))
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            got, want = _dt_both_ways(descs, probs, side)
        assert np.all(want > 0)
        np.testing.assert_array_equal(got, want)


def test_noalloc_dt_refuses_a_stream_under_capture():
    """The box table is copied from host memory that lives only for the call,
    so a graph captured around the call would keep a dangling pointer: the
    call must refuse and leave the capture intact."""
    import torch
    pr = inputs.uniform(6)
    B = hydro.Boxes([pr])
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    hydro.hydro_compute_dt_noalloc(B.descs, B.state, out)  # the per-device set-up, outside capture
    torch.cuda.synchronize()
    first = out.item()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device="cuda")
    err = None
    with torch.cuda.graph(g, stream=side):
        try:
            hydro.hydro_compute_dt_noalloc(B.descs, B.state, out, side)
        except hydro.HydroError as e:
            err = e
        x.add_(1.0)
    g.replay()
    torch.cuda.synchronize()
    assert err is not None and err.code == hydro.HYDRO_ERR_INVALID
    assert "capture" in str(err)
    assert x.cpu().tolist() == [1.0] * 4
    # still usable afterwards
    out.zero_()
    hydro.hydro_compute_dt_noalloc(B.descs, B.state, out)
    torch.cuda.synchronize()
    assert out.item() == first
    B.close()


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
