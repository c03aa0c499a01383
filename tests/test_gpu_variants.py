"""Method variants on the GPU vs the oracle with the same variant, through the
C ABI (needs a GB300): the Colella-Sekora limiter (CS08) and the two-shock
Riemann solver, alone and together.

Bars: FP64 relative L-infinity per conserved field at most 1e-10 after ten
accumulated steps on well-conditioned cases, and at most 1e-12 per step when
each step starts from the oracle's own state (every case, the ill-conditioned
ones included: see variant_cases.py); every intermediate of one step within
1e-11 of its group's scale; mixed precision at most 1e-5 relative L1 in
density and total energy; conservation to FP64 round-off.
"""
import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import domain, hydro, inputs
from test_gpu_parity import _regions, rel_linf
from variant_cases import (CASES, CS, CS_SENSITIVE, TS, VARIANTS, WELL_CONDITIONED, make_case,
                           scaled_linf)

pytestmark = pytest.mark.gpu
TOL = 1e-10
TOL_STEP = 1e-12


def run_gpu(pr, nsteps, limiter, riemann, precision=hydro.HYDRO_FP64):
    B = hydro.Boxes([pr], precision=precision, limiter=limiter, riemann=riemann)
    B.step(nsteps)
    B.sync()
    U, t = B.interior(0), B.time()[0]
    B.close()
    return U, t


@pytest.mark.parametrize("name,variant", WELL_CONDITIONED)
def test_variant_fp64_matches_oracle_after_10_steps(name, variant):
    limiter, riemann = VARIANTS[variant]
    pr = make_case(name)
    Uo, to, _, rc = oracle.run(pr, nsteps=10, nthreads=8, limiter=limiter, riemann=riemann)
    assert rc == 0
    Ug, tg = run_gpu(pr, 10, limiter, riemann)
    err = rel_linf(Ug, Uo)
    assert np.all(err <= TOL), err
    assert tg == pytest.approx(to, rel=1e-12)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("name", sorted(CASES))
def test_variant_fp64_matches_oracle_step_by_step(name, variant):
    """Ten steps, each started on the GPU from the oracle's state and dt of
    that step, so that a case's own sensitivity to rounding cannot accumulate."""
    import torch
    limiter, riemann = VARIANTS[variant]
    pr = make_case(name)
    box = oracle.box_of(pr, limiter, riemann)
    Ug = oracle.embed(pr.U)
    B = hydro.Boxes([pr], limiter=limiter, riemann=riemann)
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    worst = 0.0
    for s in range(10):
        oracle.fill_ghosts(box, Ug)
        dt = oracle.compute_dt(box, Ug)
        B.set_interior(0, oracle.interior(Ug))
        dt_dev.fill_(dt)
        rc, _ = oracle.step(box, Ug, dt, nthreads=8)
        assert rc == 0
        B.step(1, dt=dt_dev)
        B.sync()
        worst = max(worst, scaled_linf(B.interior(0), oracle.interior(Ug)))
    B.close()
    assert worst <= TOL_STEP, worst


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("name", ["sedov", "kelvin_helmholtz_reflect_y", "colliding_flows"])
def test_variant_every_stage_matches_oracle_on_one_step(name, variant):
    import torch
    limiter, riemann = VARIANTS[variant]
    pr = make_case(name)
    box = oracle.box_of(pr, limiter, riemann)
    Ug = oracle.embed(pr.U)
    oracle.fill_ghosts(box, Ug)
    dt = oracle.compute_dt(box, Ug)
    rc, W = oracle.step(box, Ug, dt, dump=True)
    assert rc == 0
    B = hydro.Boxes([pr], limiter=limiter, riemann=riemann)
    B.step(1, dt=torch.tensor([dt], dtype=torch.float64, device="cuda"))
    B.sync()
    Wg = B.field_view(0, 0, oracle.W_NFIELDS).cpu().numpy()
    Ugpu = B.interior(0)
    B.close()
    bad = []
    regions = _regions(pr.shape)
    for f, (label, reg) in regions.items():
        g0 = f if f < 5 else oracle.W_QM + (f - oracle.W_QM) // 5 * 5
        group = range(0, 5) if f < 5 else ([f] if f in (oracle.W_C, oracle.W_CHI) else range(g0, g0 + 5))
        scale = max(np.max(np.abs(W[h][regions[h][1]])) for h in group)
        diff = np.max(np.abs(Wg[f][reg] - W[f][reg]))
        if diff > 1e-11 * scale:
            bad.append((label, diff, scale))
    assert not bad, bad[:10]
    assert np.all(rel_linf(Ugpu, oracle.interior(Ug)) <= 1e-12)


MIXED_L1_PAIRS = sorted([(n, v) for n in ("sod_x", "density_wave_ragged", "kelvin_helmholtz_reflect_y")
                         for v in VARIANTS] + [("colliding_flows", "two_shock")])
# Not judged against the oracle in mixed precision (see the test below).
MIXED_UNJUDGED = sorted([("sedov", v) for v in VARIANTS] +
                        [("colliding_flows", "cs08"), ("colliding_flows", "cs08_two_shock")])


@pytest.mark.parametrize("name,variant", MIXED_L1_PAIRS)
def test_variant_mixed_matches_fp64_oracle_in_l1(name, variant):
    limiter, riemann = VARIANTS[variant]
    pr = make_case(name)
    Uo, to, _, rc = oracle.run(pr, nsteps=20, nthreads=8, limiter=limiter, riemann=riemann)
    assert rc == 0
    Um, tm = run_gpu(pr, 20, limiter, riemann, hydro.HYDRO_MIXED)
    for v in (0, 4):
        err = np.sum(np.abs(Um[v] - Uo[v])) / np.sum(np.abs(Uo[v]))
        print(f"{name} {variant} field {v}: rel L1 {err:.2e}")
        assert err <= 1e-5, (v, err)


@pytest.mark.parametrize("name,variant", MIXED_UNJUDGED)
def test_variant_mixed_conditioning_limited_cases_stay_physical(name, variant):
    """Pairs whose mixed result is not judged against the oracle in L1: on
    the Sedov blast FP32-size noise in the initial state alone moves the FP64
    oracle's own 20-step result by up to a few 1e-3 (density) and 1e-2
    (energy) in relative L1 (pinned in test_oracle_variants.py), and the
    mixed variants land anywhere in that range with ulp-level changes of the
    code (measured 6e-8 to 2e-3); under CS08 the colliding flows' symmetric
    states make second differences zero up to rounding, so FP32 rounding
    flips CS08's sign test (measured 9e-5 and 9e-4).  What must hold: every
    zone stays physical and the clock stays with the FP64 oracle's;
    conservation is checked on periodic boxes in
    test_variant_conserves_to_fp64_roundoff."""
    limiter, riemann = VARIANTS[variant]
    pr = make_case(name)
    _, to, _, rc = oracle.run(pr, nsteps=20, nthreads=8, limiter=limiter, riemann=riemann)
    assert rc == 0
    Um, tm = run_gpu(pr, 20, limiter, riemann, hydro.HYDRO_MIXED)   # raises on a nonphysical zone
    assert np.all(np.isfinite(Um)) and np.all(Um[0] > 0)
    assert tm == pytest.approx(to, rel=1e-2)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("precision", [hydro.HYDRO_FP64, hydro.HYDRO_MIXED])
def test_variant_conserves_to_fp64_roundoff(variant, precision):
    limiter, riemann = VARIANTS[variant]
    pr = inputs.kelvin_helmholtz((16, 12, 10), seed=2)
    pr.bc = ("periodic",) * 6
    U, _ = run_gpu(pr, 15, limiter, riemann, precision)
    for v in range(5):
        assert abs(U[v].sum() - pr.U[v].sum()) <= 1e-12 * np.abs(pr.U[v]).sum(), v


def test_method_can_change_between_steps():
    """The step graph is rebuilt when the method changes: 4 default steps then
    4 CS08 + two-shock steps equal the oracle doing the same."""
    pr = make_case("kelvin_helmholtz_reflect_y")
    base = oracle.box_of(pr)
    var = oracle.box_of(pr, CS, TS)
    Ug = oracle.embed(pr.U)
    t = 0.0
    for s in range(8):
        box = base if s < 4 else var
        oracle.fill_ghosts(box, Ug)
        dt = oracle.compute_dt(box, Ug)
        rc, _ = oracle.step(box, Ug, dt, nthreads=8)
        assert rc == 0
        t += dt
    B = hydro.Boxes([pr])
    B.step(4)
    hydro.hydro_set_method(B.h, CS, TS)
    B.step(4)
    B.sync()
    err = rel_linf(B.interior(0), oracle.interior(Ug))
    tg = B.time()[0]
    B.close()
    assert np.all(err <= TOL), err
    assert tg == pytest.approx(t, rel=1e-12)


def test_variant_split_domain_is_bitwise_one_box():
    pr = inputs.density_wave((24, 20, 16), seed=3)
    B = hydro.Boxes([pr], limiter=CS, riemann=TS)
    B.step(6)
    B.sync()
    whole = B.interior(0)
    B.close()
    boxes, nbr, origins = domain.decompose(pr, ([10, 14], [12, 8], [16]))
    B = hydro.Boxes(boxes, limiter=CS, riemann=TS)
    hydro.hydro_set_neighbors(B.h, nbr)
    hydro.hydro_set_shared_dt(B.h, True)
    B.step(6)
    B.sync()
    split = domain.assemble(pr.shape, [B.interior(k) for k in range(B.nboxes)], origins)
    B.close()
    np.testing.assert_array_equal(split, whole)


def test_unknown_method_codes_are_rejected():
    B = hydro.Boxes([inputs.uniform((6, 6, 6))])
    with pytest.raises(hydro.HydroError):
        hydro.hydro_set_method(B.h, 2, 0)
    with pytest.raises(hydro.HydroError):
        hydro.hydro_set_method(B.h, 0, -1)
    B.close()
