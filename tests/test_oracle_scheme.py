"""Whole-scheme pins of the oracle (CPU only): exact Riemann solutions,
conservation, symmetries, trivial states and the measured convergence order."""
import os

import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import inputs

NT = min(8, os.cpu_count() or 1)


def run_to(problem, T, nthreads=NT):
    """Advance to time T exactly (last dt clipped); returns interior U."""
    box = oracle.box_of(problem)
    Ug = oracle.embed(problem.U)
    t = 0.0
    while t < T * (1 - 1e-14):
        oracle.fill_ghosts(box, Ug)
        dt = min(oracle.compute_dt(box, Ug), T - t)
        rc, _ = oracle.step(box, Ug, dt, nthreads=nthreads)
        assert rc == 0
        t += dt
    return oracle.interior(Ug)


def sod_l1(n, T=0.15):
    pr = inputs.sod((n, 4, 4))
    U = run_to(pr, T)
    x = (np.arange(n) + 0.5) / n
    rho_ex, _, _ = oracle.riemann_sample((1, 0, 1), (0.125, 0, 0.1), 1.4, (x - 0.5) / T)
    return np.mean(np.abs(U[0, 2, 2, :] - rho_ex)), U


def test_sod_converges_to_exact_riemann_solution():
    errs = [sod_l1(n)[0] for n in (32, 64, 128)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 4e-3
    # discontinuities limit the rate to about first order
    assert np.log2(errs[0] / errs[2]) / 2 > 0.6


def test_sod_keeps_transverse_uniformity_exactly():
    _, U = sod_l1(32, T=0.1)
    assert np.all(U[2] == 0.0) and np.all(U[3] == 0.0)
    for v in range(5):
        assert np.all(U[v] == U[v][:1, :1, :])


@pytest.mark.parametrize("axis", [1, 2])
def test_sod_axis_permutation_is_exact(axis):
    px = inputs.sod((32, 4, 4), axis=0)
    shape = [4, 4, 4]
    shape[axis] = 32
    pa = inputs.sod(tuple(shape), axis=axis)
    Ux, _, dtx, rcx = oracle.run(px, nsteps=15)
    Ua, _, dta, rca = oracle.run(pa, nsteps=15)
    assert rcx == 0 and rca == 0
    np.testing.assert_array_equal(dtx, dta)
    # axis -> x: move the spatial axis of the tube to the x position and its momentum to slot 1
    perm = {1: (0, 2, 1), 2: (2, 1, 0)}[axis]  # spatial (z,y,x) axes of Ua in x-tube order
    back = np.transpose(Ua, (0,) + tuple(1 + p for p in perm))
    mom = [0, 1, 2, 3, 4]
    mom[1], mom[1 + axis] = mom[1 + axis], mom[1]
    np.testing.assert_array_equal(back[mom], Ux)


def test_sod_mirror_image():
    a = inputs.sod((48, 4, 4))
    b = inputs.sod((48, 4, 4), flip=True)
    Ua, *_ = oracle.run(a, nsteps=25)
    Ub, *_ = oracle.run(b, nsteps=25)
    mir = Ub[:, :, :, ::-1].copy()
    mir[1] *= -1
    for v in range(5):
        scale = np.max(np.abs(Ua[v])) or 1.0
        assert np.max(np.abs(mir[v] - Ua[v])) <= 1e-12 * scale


@pytest.mark.parametrize("bc", ["periodic", "outflow", "reflect"])
def test_uniform_state_stays_uniform(bc):
    vel = (0.3, -0.2, 0.1) if bc != "reflect" else (0.0, 0.0, 0.0)
    pr = inputs.uniform((8, 6, 5), vel=vel, bc=bc)
    U, *_ = oracle.run(pr, nsteps=6)
    for v in range(5):
        np.testing.assert_allclose(U[v], pr.U[v], rtol=1e-14, atol=1e-15)


def test_stationary_contact_is_exact():
    pr = inputs.uniform((16, 4, 4), vel=(0, 0, 0), p=1.0, bc="outflow")
    pr.U[0, :, :, 8:] = 0.1  # density jump, same pressure, at rest
    U, *_ = oracle.run(pr, nsteps=10)
    np.testing.assert_array_equal(U, pr.U)


def _conserved_drift(pr, nsteps):
    U0 = pr.U
    U, t, dts, rc = oracle.run(pr, nsteps=nsteps, nthreads=NT)
    assert rc == 0
    drift = [abs(U[v].sum() - U0[v].sum()) / np.abs(U0[v]).sum() for v in range(5)]
    return np.array(drift)


def test_conservation_periodic_density_wave():
    pr = inputs.density_wave((12, 10, 8), seed=7)
    nsteps = 10
    assert np.all(_conserved_drift(pr, nsteps) <= 1e-13 * np.sqrt(nsteps))


def test_conservation_periodic_shear_layer():
    pr = inputs.kelvin_helmholtz(12, seed=2)
    pr.bc = ("periodic",) * 6
    nsteps = 10
    assert np.all(_conserved_drift(pr, nsteps) <= 1e-13 * np.sqrt(nsteps))


def test_reflecting_walls_conserve_mass_energy_and_tangential_momentum():
    pr = inputs.kelvin_helmholtz(12, seed=2)  # reflect in y
    U0 = pr.U
    U, *_ = oracle.run(pr, nsteps=8, nthreads=NT)
    for v in (0, 1, 3, 4):
        assert abs(U[v].sum() - U0[v].sum()) <= 1e-13 * np.sqrt(8) * np.abs(U0[v]).sum()


def test_reflecting_wall_fluxes_are_impermeable():
    pr = inputs.kelvin_helmholtz((8, 10, 6), seed=3)
    box = oracle.box_of(pr)
    Ug = oracle.embed(pr.U)
    oracle.fill_ghosts(box, Ug)
    rc, W = oracle.step(box, Ug, oracle.compute_dt(box, Ug), dump=True)
    g, ny = 4, 10
    for wall in (g, g + ny):  # y faces at j = 0 and j = ny
        F = W[oracle.W_F + 5 * 1:oracle.W_F + 5 * 2, g:-g, wall, g:-g]
        assert np.all(F[[0, 1, 3, 4]] == 0.0)
        assert np.all(F[2] > 0.0)  # the wall pressure


def test_shear_layer_mirror_symmetry_about_midplane():
    a = inputs.kelvin_helmholtz(12, seed=5)
    b = inputs.kelvin_helmholtz(12, seed=5)
    b.U = a.U[:, :, ::-1, :].copy()
    b.U[2] *= -1
    Ua, *_ = oracle.run(a, nsteps=6, nthreads=NT)
    Ub, *_ = oracle.run(b, nsteps=6, nthreads=NT)
    mir = Ub[:, :, ::-1, :].copy()
    mir[2] *= -1
    for v in range(5):
        scale = np.max(np.abs(Ua[v]))
        assert np.max(np.abs(mir[v] - Ua[v])) <= 1e-12 * scale


def test_sedov_axis_permutation_symmetry():
    a = inputs.sedov((16, 16, 16), seed=1)
    b = inputs.sedov((16, 16, 16), seed=1)
    b.U = np.transpose(a.U, (0, 1, 3, 2))[[0, 2, 1, 3, 4]].copy()  # swap x and y
    Ua, *_ = oracle.run(a, nsteps=8, nthreads=NT)
    Ub, *_ = oracle.run(b, nsteps=8, nthreads=NT)
    back = np.transpose(Ub, (0, 1, 3, 2))[[0, 2, 1, 3, 4]]
    for v in range(5):
        scale = np.max(np.abs(Ua[v]))
        assert np.max(np.abs(back[v] - Ua[v])) <= 1e-12 * scale


def test_sedov_blast_stays_centred_and_expands():
    pr = inputs.sedov((24, 24, 24), seed=3)
    ci, cj, ck = pr.meta["centre"]
    U, t, *_ = oracle.run(pr, nsteps=20, nthreads=NT)
    rho = U[0]
    k, j, i = np.meshgrid(*(np.arange(24),) * 3, indexing="ij")
    r = np.sqrt((i - ci) ** 2 + (j - cj) ** 2 + (k - ck) ** 2) / 64.0
    # shell of peak density: Sedov-Taylor radius xi0 (E t^2/rho)^(1/5), xi0 ~ 1.03-1.15 (gamma 1.4)
    r_shell = np.sum(r * (rho > 1.5)) / max(1, np.sum(rho > 1.5))
    r_st = (1.0 * t * t) ** 0.2
    assert 0.7 * r_st < r_shell < 1.4 * r_st


def _wave_error(n, T=0.05):
    pr = inputs.density_wave(n, noise=0.0)
    U = run_to(pr, T)
    x = (np.arange(n) + 0.5) / n
    X = x[None, None, :] + x[None, :, None] + x[:, None, None]
    exact = 1 + 0.1 * np.sin(2 * np.pi * (X - 1.75 * T))
    return np.mean(np.abs(U[0] - exact))


def test_smooth_wave_converges_at_second_order():
    e16, e32 = _wave_error(16), _wave_error(32)
    assert np.log2(e16 / e32) >= 1.8


@pytest.mark.slow
def test_smooth_wave_converges_at_second_order_64():
    e32, e64 = _wave_error(32), _wave_error(64)
    assert np.log2(e32 / e64) >= 1.8


def test_nonphysical_initial_state_is_reported():
    pr = inputs.uniform(8, bc="periodic")
    pr.U[0, 3, 3, 3] = -1.0
    U, t, dts, rc = oracle.run(pr, nsteps=2)
    assert rc == -3


def test_invalid_box_is_rejected():
    pr = inputs.uniform(8)
    pr.bc = ("periodic", "outflow", "periodic", "periodic", "periodic", "periodic")
    with pytest.raises(ValueError):
        oracle.run(pr, nsteps=1)
