"""Pins of the oracle's corner-transport constants, its guard branches and the
flattening constants (CPU only).

- The 3D CTU stages (Colella 1990; Saltzman 1994): for a density checkerboard
  carried by a uniform velocity at uniform pressure, every zone is a local
  extremum along every axis, so the CW84 limiter reconstructs each zone as a
  constant, HLLC resolves the contact exactly (F = rho_upwind u), and a step
  reduces to the linear first-order CTU scheme.  With stage-1 factor
  dt/(3 dx_e), stage-2 factor dt/(2 dx_e) and stage 2 correcting a d-face by
  the fluxes of the pairs (e|f) and (f|e), that scheme is exactly the product
  of the three 1D upwind operators, (1 - X)(1 - Y)(1 - Z) with X = sigma_x
  times the upwind difference along x; on the checkerboard each factor is the
  number 1 - 2 sigma_d.  Any other factor or pairing changes the
  coefficients of XY, XZ, YZ or XYZ and with them the amplitude.
- R11: with the wall override off, the flux through a reflecting face still
  carries mass and energy at round-off only (its two states are mirror
  images), so R11 changes FP64 results by rounding alone.
- Guard branches: the inputs the GPU parity cases use for them do reach them.
- Flattening constants: hand-worked CW84 coefficients (tests/golden).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import inputs

GOLDEN_FLAT = os.path.join(os.path.dirname(__file__), "golden", "cw84_flattening.txt")

CHECKER_CASES = [((1.0, -0.6, 0.35), 0.9), ((0.3, 0.8, -0.5), 0.6), ((-1.0, 1.0, 1.0), 0.95),
                 ((0.7, 0.0, 0.2), 0.5), ((0.45, -0.45, 0.9), 0.75)]


def _parity_sign(shape):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return 1.0 - 2.0 * ((i + j + k) % 2)


@pytest.mark.parametrize("vel,cfl", CHECKER_CASES)
def test_ctu_step_on_a_checkerboard_is_the_product_of_1d_upwind_factors(vel, cfl):
    pr = inputs.checkerboard((8, 6, 4), vel=vel, cfl=cfl)
    box = oracle.box_of(pr)
    Ug = oracle.embed(pr.U)
    sgn = _parity_sign(pr.U.shape[1:])
    rho0, amp, p, g = pr.meta["rho0"], pr.meta["amp"], pr.meta["p"], pr.gamma
    for _ in range(4):
        oracle.fill_ghosts(box, Ug)
        dt = oracle.compute_dt(box, Ug)
        rc, _ = oracle.step(box, Ug, dt)
        assert rc == 0
        sig = [abs(vel[d]) * dt / pr.dx[d] for d in range(3)]
        amp *= np.prod([1.0 - 2.0 * s for s in sig])
        U = oracle.interior(Ug)
        rho = rho0 + amp * sgn
        np.testing.assert_allclose(U[0], rho, rtol=0, atol=2e-14)
        for d in range(3):
            np.testing.assert_allclose(U[1 + d], vel[d] * rho, rtol=0, atol=2e-14)
        np.testing.assert_allclose(U[4], p / (g - 1.0) + 0.5 * np.dot(vel, vel) * rho, rtol=0, atol=2e-14)


def test_ctu_checkerboard_stays_bounded_up_to_cfl_one():
    """|1 - 2 sigma| <= 1 for every sigma in [0, 1]: the full 3D CTU keeps the
    checkerboard bounded at Courant numbers up to 1 along every axis at once
    (a 6-solve variant without the stage-2 cross terms is not stable there)."""
    pr = inputs.checkerboard((6, 6, 6), vel=(1.0, 1.0, 1.0), p=1e-4, cfl=1.0, nsteps=60)
    U, t, dts, rc = oracle.run(pr)
    assert rc == 0
    sgn = _parity_sign(U.shape[1:])
    amp = float(np.mean((U[0] - 1.0) * sgn))
    expect = 0.1 * np.prod([(1.0 - 2.0 * dt * 6.0) ** 3 for dt in dts])
    assert abs(amp) <= 0.1
    # rounding of the decaying amplitude accumulates over the 60 steps; a wrong
    # CTU factor changes the factor per step by order one (and grows it past 1)
    assert abs(amp - expect) <= 1e-8 * abs(expect)


def test_r11_changes_fp64_results_by_rounding_alone():
    pr = inputs.kelvin_helmholtz((10, 12, 8), seed=5, nsteps=8)
    box = oracle.box_of(pr)
    try:
        oracle.set_wall_r11(False)
        Ug = oracle.embed(pr.U)
        fmax = 0.0
        for _ in range(pr.nsteps):
            oracle.fill_ghosts(box, Ug)
            dt = oracle.compute_dt(box, Ug)
            rc, W = oracle.step(box, Ug, dt, dump=True)
            assert rc == 0
            F = W[oracle.W_F + 5:oracle.W_F + 10]  # y-fluxes (conserved x,y,z order)
            g = oracle.NG
            ny = pr.shape[1]
            for jw in (0, ny):  # the faces at y = 0 and y = n_y, stored at their high-side zone
                walls = F[:, g:-g, g + jw, g:-g]
                scale = np.max(np.abs(F[2, g:-g, g:-g, g:-g]))
                for v in (0, 1, 3, 4):  # mass, tangential momenta, energy
                    fmax = max(fmax, float(np.max(np.abs(walls[v]))) / scale)
        U_off = oracle.interior(Ug)
    finally:
        oracle.set_wall_r11(True)
    U_on, *_ = oracle.run(pr)
    assert fmax <= 1e-14
    for v in range(5):
        scale = np.max(np.abs(U_on[v])) or 1.0
        assert np.max(np.abs(U_off[v] - U_on[v])) <= 1e-13 * scale


def test_hllc_takes_the_davis_bounds_only_where_rounding_hides_the_sound_speed_and_stays_consistent():
    """The Roe sound speed squared is a sum of non-negative terms for any
    physical pair of states, so the Davis fallback can only be reached when
    rounding of the kinetic energy swamps the enthalpy (Mach ~ 1e8 and
    beyond); there HLLC must still return the physical flux of equal states."""
    oracle.branch_hits(reset=True)
    q = np.array([1.0, 1e4, 0.0, 0.0, 1e-12])
    F = oracle.hllc(0, q, q, 1.4)
    assert oracle.branch_hits()["davis"] == 1
    E = q[4] / 0.4 + 0.5 * q[0] * q[1] ** 2
    np.testing.assert_allclose(F, [q[0] * q[1], q[0] * q[1] ** 2 + q[4], 0.0, 0.0, (E + q[4]) * q[1]],
                               rtol=1e-15)
    q2 = np.array([1.0, 10.0, 0.5, 0.0, 1e-3])
    oracle.hllc(0, q2, q2 * [1.1, 1.0, 1.0, 1.0, 0.9], 1.4)
    assert oracle.branch_hits()["davis"] == 0


def test_tracing_floors_a_state_below_the_density_and_pressure_floors():
    n = 12
    q = np.zeros((5, n))
    q[0] = 1e-13
    q[4] = np.where(np.arange(n) < n // 2, 1e-13, 5e-14)
    c = np.sqrt(1.4 * q[4] / q[0])
    oracle.branch_hits(reset=True)
    qm, qp = oracle.trace_line(q, c, np.zeros(n), 0.5 / np.max(c))
    hits = oracle.branch_hits()
    assert hits["trace_dens_floor"] > 0 and hits["trace_pres_floor"] > 0
    assert np.all(qm[0, 2:-2] == 1e-12) and np.all(qp[4, 2:-2] == 1e-12)


def test_cold_blast_reaches_the_pressure_floors():
    """Sedov blast into an ambient pressure (1e-14) below the floor: every
    ambient zone's primitive pressure is floored, and so is a corrected state
    at the front."""
    pr = inputs.sedov((16, 16, 16), p_ambient=1e-14, nsteps=10)
    oracle.branch_hits(reset=True)
    U, t, dts, rc = oracle.run(pr)
    hits = oracle.branch_hits()
    assert rc == 0 and np.all(np.isfinite(U))
    assert hits["prim_pres_floor"] > 0


def test_gas_ball_in_vacuum_reaches_the_density_floor():
    pr = inputs.vacuum_ball((16, 16, 16), nsteps=10)
    oracle.branch_hits(reset=True)
    U, t, dts, rc = oracle.run(pr)
    hits = oracle.branch_hits()
    assert rc == 0 and np.all(np.isfinite(U))
    assert hits["prim_dens_floor"] > 0 and hits["prim_pres_floor"] > 0


def test_revert_rule_keeps_the_cold_shear_physical():
    """Large velocity noise at low pressure: some transversely corrected
    face states come out with p <= 0 in both CTU stages; keeping the
    uncorrected state (R6) is what keeps the step physical."""
    pr = inputs.shear_cold()
    oracle.branch_hits(reset=True)
    U, t, dts, rc = oracle.run(pr)
    hits = oracle.branch_hits()
    assert rc == 0 and np.all(np.isfinite(U))
    assert hits["revert_stage1"] > 0 and hits["revert_stage2"] > 0


def _golden_flat():
    rows = []
    for line in open(GOLDEN_FLAT):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows.append((parts[0], np.array(parts[1:12], dtype=float), np.array(parts[12:17], dtype=float)))
    return rows


@pytest.mark.parametrize("name,p,f", _golden_flat(), ids=[r[0] for r in _golden_flat()])
def test_flattening_coefficients_match_hand_worked_cw84_values(name, p, f):
    got = oracle.flatten_line(p, -0.1 * np.arange(p.size))
    np.testing.assert_allclose(got[3:8], f, rtol=0, atol=1e-12)
