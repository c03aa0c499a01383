"""GPU parity on the method's guard branches and on the CTU closed form
(needs a GB300; calls through the C ABI).

- A density checkerboard carried by a uniform velocity reduces the scheme to
  the first-order 3D CTU, whose amplitude factor per step is the product of
  the three 1D upwind factors 1 - 2 sigma_d (the oracle's pin of the CTU
  constants): the FP64 path must reproduce it, and the mixed form to FP32
  rounding.
- Cases that reach the primitive-state floors (a blast into gas below the
  pressure floor, a gas ball in a near vacuum below both floors) and the CTU
  revert rule in both stages (a low-pressure shear layer with large velocity
  noise): the oracle run that serves as reference counts the branch hits,
  and each test asserts that its branch was taken there.  FP64 against the
  oracle at 1e-10 relative L-inf after 10 steps; mixed precision at 1e-5
  relative L1 in rho and E.
- A subnormal momentum, which sends the integer-pipe FP64 products that read
  it to the recomputation with the FP64 multiply, with either Riemann
  solver.
"""
import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10
TOL_L1 = 1e-5


def rel_linf(a, b):
    out = []
    for v in range(a.shape[0]):
        scale = np.max(np.abs(b[v]))
        out.append(np.max(np.abs(a[v] - b[v])) / scale if scale > 0 else np.max(np.abs(a[v] - b[v])))
    return np.array(out)


def rel_l1(a, b):
    return np.sum(np.abs(a - b)) / np.sum(np.abs(b))


def run_gpu(pr, nsteps, precision):
    B = hydro.Boxes([pr], precision=precision)
    B.step(nsteps)
    B.sync()
    out, t = B.interior(0), B.time()[0]
    B.close()
    return out, t


def _parity_sign(shape):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return 1.0 - 2.0 * ((i + j + k) % 2)


@pytest.mark.parametrize("vel,cfl", [((1.0, -0.6, 0.35), 0.9), ((-1.0, 1.0, 1.0), 0.95), ((0.3, 0.8, -0.5), 0.6)])
@pytest.mark.parametrize("precision", [hydro.HYDRO_FP64, hydro.HYDRO_MIXED])
def test_checkerboard_amplitude_is_the_product_of_1d_upwind_factors(vel, cfl, precision):
    import torch
    pr = inputs.checkerboard((16, 10, 8), vel=vel, cfl=cfl)
    B = hydro.Boxes([pr], precision=precision)
    sgn = _parity_sign(pr.U.shape[1:])
    amp = pr.meta["amp"]
    tol = 2e-14 if precision == hydro.HYDRO_FP64 else 1e-6
    for _ in range(4):
        dt = B.compute_dt().clone()
        B.step(1, dt=dt)
        B.sync()
        dtv = float(dt.cpu()[0])
        amp *= np.prod([1.0 - 2.0 * abs(vel[d]) * dtv / pr.dx[d] for d in range(3)])
        U = B.interior(0)
        rho = pr.meta["rho0"] + amp * sgn
        np.testing.assert_allclose(U[0], rho, rtol=0, atol=tol)
        for d in range(3):
            np.testing.assert_allclose(U[1 + d], vel[d] * rho, rtol=0, atol=tol)
    torch.cuda.synchronize()
    B.close()


EDGE_CASES = {
    # branch that the case must reach in the oracle run -> maker
    "cold_blast": (("prim_pres_floor",), lambda: inputs.sedov((16, 16, 16), p_ambient=1e-14, nsteps=10)),
    "vacuum_ball": (("prim_dens_floor", "prim_pres_floor"), lambda: inputs.vacuum_ball((16, 16, 16), nsteps=10)),
    "shear_cold_revert": (("revert_stage1", "revert_stage2"), lambda: inputs.shear_cold()),
}


@pytest.mark.parametrize("name", sorted(EDGE_CASES))
def test_fp64_matches_oracle_on_guard_branches(name):
    branches, make = EDGE_CASES[name]
    pr = make()
    oracle.branch_hits(reset=True)
    Uo, to, _, rc = oracle.run(pr, nsteps=10)
    hits = oracle.branch_hits()
    assert rc == 0
    for br in branches:
        assert hits[br] > 0, (br, hits)
    Ug, tg = run_gpu(pr, 10, hydro.HYDRO_FP64)
    err = rel_linf(Ug, Uo)
    assert np.all(err <= TOL), err
    assert tg == pytest.approx(to, rel=1e-12)


@pytest.mark.parametrize("name", sorted(EDGE_CASES))
def test_mixed_matches_oracle_on_guard_branches(name):
    branches, make = EDGE_CASES[name]
    pr = make()
    oracle.branch_hits(reset=True)
    Uo, to, _, rc = oracle.run(pr, nsteps=10)
    hits = oracle.branch_hits()
    assert rc == 0
    for br in branches:
        assert hits[br] > 0, (br, hits)
    Um, tm = run_gpu(pr, 10, hydro.HYDRO_MIXED)
    err_rho, err_E = rel_l1(Um[0], Uo[0]), rel_l1(Um[4], Uo[4])
    print(f"{name}: rel L1 rho {err_rho:.3e}, E {err_E:.3e}")
    assert err_rho <= TOL_L1 and err_E <= TOL_L1, (err_rho, err_E)


@pytest.mark.parametrize("riemann", [hydro.HYDRO_RIEMANN_HLLC, hydro.HYDRO_RIEMANN_TWO_SHOCK])
def test_subnormal_momentum_takes_the_fp64_multiply_recomputation(riemann):
    # A transverse velocity of 1e-310 makes that momentum subnormal: every
    # integer-pipe product that reads it (the primitive conversion's m / rho,
    # the conserved form of each traced state, the corrections' velocities,
    # the Riemann solvers' transverse fluxes) defers, and the warps redo those
    # units with the FP64 multiply.  The result must still match the oracle.
    pr = inputs.density_wave((24, 20, 16), seed=2, vel=(1.0, 0.5, 1e-310))
    assert 0.0 < np.max(np.abs(pr.U[3])) < 2.2250738585072014e-308  # subnormal
    Uo, to, _, rc = oracle.run(pr, nsteps=10, nthreads=8, riemann=riemann)
    assert rc == 0
    B = hydro.Boxes([pr], riemann=riemann)
    B.step(10)
    B.sync()
    U, t = B.interior(0), B.time()[0]
    B.close()
    err = rel_linf(U, Uo)
    print("rel L-inf per field", err)
    assert np.all(err <= TOL), err
    assert t == pytest.approx(to, rel=1e-12)
