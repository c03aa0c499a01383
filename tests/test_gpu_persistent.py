"""The persistent form (hydro_persistent): one launch advances every box by all
steps, its blocks taking stage work from a queue with bounded per-box waits
(needs a GB300; through the C ABI).

- The stage work is the per-stage kernels' own code, so a run in the
  persistent form equals the per-stage form bit for bit, for FP64 and mixed
  boxes of uneven sizes, with dt from the state or given, and for the method
  variants.
- A wait that can never be met (the test hook stall_box) gives up after the
  spin limit: the launch ends by itself, hydro_sync reports HYDRO_ERR_TIMEOUT,
  and the handle keeps working afterwards.
"""
import numpy as np
import pytest

from paper_2007_05218_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu


def run(problems, nsteps, persistent, precision=hydro.HYDRO_FP64, limiter=0, riemann=0, dt=None):
    import torch
    B = hydro.Boxes(problems, precision=precision, limiter=limiter, riemann=riemann)
    if persistent:
        hydro.hydro_persistent(B.h, True)
    dt_dev = None if dt is None else torch.tensor(dt, dtype=torch.float64, device="cuda")
    B.step(nsteps, dt=dt_dev)
    B.sync()
    out = [B.interior(b) for b in range(B.nboxes)]
    t = B.time()
    B.close()
    return out, t


@pytest.mark.parametrize("precision", [hydro.HYDRO_FP64, hydro.HYDRO_MIXED])
def test_persistent_form_equals_the_per_stage_form_bitwise(precision):
    probs = inputs.sedov_batch(9, seed=5, nsteps=4, edges=(12, 16, 24, 32))
    a, ta = run(probs, 4, True, precision)
    b, tb = run(probs, 4, False, precision)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(ta, tb)


def test_persistent_form_equals_the_per_stage_form_bitwise_over_many_steps():
    # Sedov boxes of the 512-box batch, past the step where the blast front's
    # far field first reaches tiny momenta: two compiled copies of a stage body
    # that round one product differently drift apart there by an ulp
    probs = inputs.sedov_batch(512, seed=0, nsteps=30)[:32]
    a, ta = run(probs, 12, True)
    b, tb = run(probs, 12, False)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(ta, tb)


def test_persistent_form_one_large_box_and_given_dt():
    pr = inputs.kelvin_helmholtz((40, 48, 36), seed=3)
    (a,), ta = run([pr], 3, True, dt=[2e-4])
    (b,), tb = run([pr], 3, False, dt=[2e-4])
    np.testing.assert_array_equal(a, b)
    assert ta[0] == tb[0] == pytest.approx(6e-4)


@pytest.mark.parametrize("limiter,riemann", [(hydro.HYDRO_LIMITER_CS08, hydro.HYDRO_RIEMANN_HLLC),
                                             (hydro.HYDRO_LIMITER_CW84, hydro.HYDRO_RIEMANN_TWO_SHOCK)])
def test_persistent_form_method_variants(limiter, riemann):
    probs = [inputs.sod((40, 6, 5), axis=0), inputs.density_wave((16, 12, 10), seed=2)]
    for prec in (hydro.HYDRO_FP64, hydro.HYDRO_MIXED):
        a, _ = run(probs, 3, True, prec, limiter, riemann)
        b, _ = run(probs, 3, False, prec, limiter, riemann)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_a_wait_that_cannot_be_met_gives_up_and_reports_a_timeout():
    import time
    probs = inputs.sedov_batch(4, seed=7, nsteps=2, edges=(16, 24))
    B = hydro.Boxes(probs)
    hydro.hydro_persistent(B.h, True)
    hydro.hydro_set_spin_limit(B.h, 4000, stall_box=1)
    t0 = time.perf_counter()
    B.step(2)
    with pytest.raises(hydro.HydroError) as e:
        B.sync()
    assert e.value.code == hydro.HYDRO_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the handle still works: restore the initial state and run normally
    hydro.hydro_set_spin_limit(B.h, 1 << 22, stall_box=-1)
    for k, p in enumerate(probs):
        B.set_interior(k, p.U)
    B.step(2)
    B.sync()
    got = [B.interior(k) for k in range(B.nboxes)]
    B.close()
    ref, _ = run(probs, 2, False)
    for x, y in zip(got, ref):  # the interrupted step left nothing behind that changes the next ones
        np.testing.assert_array_equal(x, y)


def test_persistent_form_refuses_linked_boxes_and_tiles():
    probs = [inputs.uniform((8, 8, 8)), inputs.uniform((8, 8, 8))]
    B = hydro.Boxes(probs, precision=hydro.HYDRO_MIXED)
    hydro.hydro_fuse_tiles(B.h, True)
    with pytest.raises(hydro.HydroError):
        hydro.hydro_persistent(B.h, True)
    hydro.hydro_fuse_tiles(B.h, False)
    hydro.hydro_persistent(B.h, True)
    with pytest.raises(hydro.HydroError):
        hydro.hydro_set_neighbors(B.h, np.array([[-1, 1, -1, -1, -1, -1], [0, -1, -1, -1, -1, -1]]))
    with pytest.raises(hydro.HydroError):
        hydro.hydro_autotune(B.h, reps=1)
    hydro.hydro_persistent(B.h, False)
    B.close()
