"""Pins of the oracle's method variants (CPU only): the Colella-Sekora
extremum-preserving limiter (CS08) and the two-shock Riemann solver (Colella &
Glaz 1985).  Each pin rests on mathematics or on printed values, never on the
oracle itself: exactness on polynomials, measured orders of accuracy, exact
Riemann solutions (pinned to Toro's table in test_oracle_riemann.py and to the
golden file read here), closed forms, symmetries."""
import os

import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import inputs

NT = min(8, os.cpu_count() or 1)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toro_riemann_star.txt")
GAMMA = 1.4


def cell_averages(poly, n, h, x0):
    """Exact averages over [x0 + i h, x0 + (i+1) h] of a polynomial (numpy
    coefficient order) and the zone edges."""
    P = np.polyint(poly)
    e = x0 + h * np.arange(n + 1)
    return (np.polyval(P, e[1:]) - np.polyval(P, e[:-1])) / h, e


# ---------------------------------------------------------------- CS08 limiter
@pytest.mark.parametrize("seed", range(6))
def test_cs_parabolas_are_exact_for_quadratics_even_at_the_extremum(seed):
    """CS08's purpose: a smooth extremum is not clipped.  The averages of a
    quadratic give its exact edge values in every zone, the one holding the
    extremum included, while the CW84 limiter flattens that zone."""
    rng = np.random.default_rng(seed)
    n, h = 24, 0.1
    poly = rng.normal(size=3)
    vertex = -poly[1] / (2 * poly[0])
    x0 = vertex - (n // 2 + rng.uniform(0, 1)) * h   # the extremum inside the line
    a, e = cell_averages(poly, n, h, x0)
    aL, aR = oracle.ppm_line_cs(a)
    s = slice(2, n - 2)
    scale = np.max(np.abs(a))
    assert np.max(np.abs(aL[s] - np.polyval(poly, e[:-1])[s])) <= 1e-13 * scale
    assert np.max(np.abs(aR[s] - np.polyval(poly, e[1:])[s])) <= 1e-13 * scale
    bL, _ = oracle.ppm_line(a)
    assert np.max(np.abs(bL[s] - np.polyval(poly, e[:-1])[s])) > 1e-6 * scale


def test_cs_parabolas_are_exact_for_a_monotone_cubic():
    """The 4th-order interface interpolant is exact for cubics; on monotone
    data neither limiter step changes it."""
    poly = np.array([1.0, 0.0, 1.0, 0.3])   # x^3 + x + 0.3, increasing everywhere
    a, e = cell_averages(poly, 24, 0.05, -0.6)
    aL, aR = oracle.ppm_line_cs(a)
    s = slice(2, 22)
    np.testing.assert_allclose(aL[s], np.polyval(poly, e[:-1])[s], rtol=0, atol=1e-14)
    np.testing.assert_allclose(aR[s], np.polyval(poly, e[1:])[s], rtol=0, atol=1e-14)


def _sine_edge_error(N, line):
    h = 1.0 / N
    x = np.arange(-4, N + 4) * h
    a = (np.cos(2 * np.pi * x) - np.cos(2 * np.pi * (x + h))) / (2 * np.pi * h)  # averages of sin(2 pi x)
    aL, _ = line(a)
    s = slice(4, N + 4)
    return np.max(np.abs(aL[s] - np.sin(2 * np.pi * x[s])))


def test_cs_edge_values_converge_at_high_order_through_extrema():
    """Maximum edge error over a sine wave (two extrema): CS08 keeps the
    interpolant's high order (at least third) through the extrema; CW84 drops
    to second order there."""
    cs = [_sine_edge_error(N, oracle.ppm_line_cs) for N in (32, 64, 128)]
    cw = [_sine_edge_error(N, oracle.ppm_line) for N in (32, 64, 128)]
    assert np.log2(cs[0] / cs[2]) / 2 >= 3.0
    assert 1.8 <= np.log2(cw[0] / cw[2]) / 2 <= 2.2
    assert cs[2] < 1e-3 * cw[2]


@pytest.mark.parametrize("seed", range(4))
def test_cs_makes_no_new_extrema_at_discontinuities(seed):
    """Piecewise-constant data (plateaus of five zones, random jumps): every
    edge value lies between the two zone values that share the edge."""
    rng = np.random.default_rng(seed)
    a = np.repeat(rng.normal(size=10), 5)
    aL, aR = oracle.ppm_line_cs(a)
    i = np.arange(2, a.size - 2)
    tol = 1e-15
    assert np.all(aL[i] >= np.minimum(a[i - 1], a[i]) - tol)
    assert np.all(aL[i] <= np.maximum(a[i - 1], a[i]) + tol)
    assert np.all(aR[i] >= np.minimum(a[i + 1], a[i]) - tol)
    assert np.all(aR[i] <= np.maximum(a[i + 1], a[i]) + tol)


def test_cs_curvature_bound_worked_case():
    """A cusp worked by hand from CS08's definitions, where the bound C = 1.25
    is what limits: zone values (-6, -3, -1, 0, -1, -3, -6), middle zone 3.
    Interfaces: 7/12 (0 - 1) - 1/12 (-1 - 3) = -1/4 on both sides (inside
    their bounds).  Parabola curvature 6 (-1/4 - 1/4 - 0) = -3; neighbouring
    second differences -1, -2, -1 share its sign, so it is cut to
    -C * 1 = -1.25 and both edges move to 0 + (-1/4)(1.25/3) = -5/48."""
    a = np.array([-6.0, -3.0, -1.0, 0.0, -1.0, -3.0, -6.0])
    aL, aR = oracle.ppm_line_cs(a)
    assert aL[3] == pytest.approx(-5.0 / 48.0, rel=1e-14)
    assert aR[3] == pytest.approx(-5.0 / 48.0, rel=1e-14)


def test_cs_full_flattening_gives_the_zone_value():
    rng = np.random.default_rng(3)
    a = rng.normal(size=20)
    aL, aR = oracle.ppm_line_cs(a, np.ones_like(a))
    np.testing.assert_array_equal(aL[2:-2], a[2:-2])
    np.testing.assert_array_equal(aR[2:-2], a[2:-2])


# ------------------------------------------------------------ two-shock solver
def _golden_rows():
    rows = np.loadtxt(GOLDEN)
    return rows


def _shock_shock(row):
    """Rows of Toro's table whose star pressure exceeds both initial pressures
    (both waves are shocks)."""
    return row[6] > row[2] and row[6] > row[5]


def test_two_shock_reproduces_toros_table_when_both_waves_are_shocks():
    """With two shocks the Hugoniot is the exact wave curve, so the two-shock
    star state is the exact one: Toro's Table 4.3 test 5, all four values.
    The star densities are sampled by a Galilean shift that puts x/t = 0 just
    left, then just right, of the contact."""
    rows = [r for r in _golden_rows() if _shock_shock(r)]
    assert rows
    for r in rows:
        rl, ul, pl, rr, ur, pr, ps, us, rsl, rsr = r
        L = np.array([rl, ul, 0.0, 0.0, pl])
        R = np.array([rr, ur, 0.0, 0.0, pr])
        p_star, u_star, _, _, _ = oracle.two_shock(L, R, GAMMA)
        assert p_star == pytest.approx(ps, rel=5e-5)
        assert u_star == pytest.approx(us, rel=5e-5)
        for shift, rho_expect in ((-1e-3, rsl), (1e-3, rsr)):
            Ls, Rs = L.copy(), R.copy()
            Ls[1] -= u_star + shift
            Rs[1] -= u_star + shift
            _, _, q, _, _ = oracle.two_shock(Ls, Rs, GAMMA)
            assert q[0] == pytest.approx(rho_expect, rel=5e-5)


@pytest.mark.parametrize("seed", range(5))
def test_two_shock_equals_the_exact_solver_for_colliding_flows(seed):
    """Random colliding states (both waves shocks in the exact solution): star
    values and the state at x/t = 0 equal the exact solver's."""
    rng = np.random.default_rng(seed)
    for _ in range(20):
        rl, rr = rng.uniform(0.2, 5.0, 2)
        pl, pr = rng.uniform(0.1, 10.0, 2)
        ul = rng.uniform(-3.0, 3.0)
        ur = ul - rng.uniform(1.0, 8.0)
        pe, ue = oracle.riemann_star((rl, ul, pl), (rr, ur, pr), GAMMA)
        if not (pe > pl and pe > pr):
            continue
        L = np.array([rl, ul, 0.4, -0.1, pl])
        R = np.array([rr, ur, -0.3, 0.2, pr])
        p_star, u_star, q, F, _ = oracle.two_shock(L, R, GAMMA)
        assert p_star == pytest.approx(pe, rel=1e-11)
        assert u_star == pytest.approx(ue, rel=1e-11, abs=1e-11 * abs(ul - ur))
        rho0, u0, p0 = oracle.riemann_sample((rl, ul, pl), (rr, ur, pr), GAMMA, np.array([0.0]))
        assert q[0] == pytest.approx(rho0[0], rel=1e-10)
        assert q[1] == pytest.approx(u0[0], rel=1e-10, abs=1e-10 * abs(ul - ur))
        assert q[4] == pytest.approx(p0[0], rel=1e-10)
        # transverse velocities ride with the material on the upwind side
        assert tuple(q[2:4]) == (tuple(L[2:4]) if u_star >= 0 else tuple(R[2:4]))


@pytest.mark.parametrize("u0", [0.5, 2.0, 10.0])
def test_two_shock_symmetric_collision_and_expansion_closed_form(u0):
    """Equal states meeting at +-u0: u* = 0 and (p* - p0)^2 = u0^2 W^2 with
    W^2 = rho ((gamma+1)/2 p* + (gamma-1)/2 p0), a quadratic in p* - p0 whose
    positive root is the collision and negative root the expansion (floored
    at the pressure floor when it would be negative)."""
    rho, p0 = 1.3, 0.7
    b = (GAMMA + 1) * u0 * u0 * rho / 2
    disc = np.sqrt(b * b + 4 * GAMMA * p0 * u0 * u0 * rho)
    p_col, u_col, q, F, _ = oracle.two_shock([rho, u0, 0, 0, p0], [rho, -u0, 0, 0, p0], GAMMA)
    assert p_col == pytest.approx(p0 + (b + disc) / 2, rel=1e-13)
    assert u_col == 0.0
    assert F[0] == 0.0 and F[1] == pytest.approx(p_col, rel=1e-13)
    p_exp, u_exp, _, _, _ = oracle.two_shock([rho, -u0, 0, 0, p0], [rho, u0, 0, 0, p0], GAMMA)
    assert p_exp == pytest.approx(max(p0 + (b - disc) / 2, 1e-12), rel=1e-12)
    assert u_exp == 0.0


def test_two_shock_star_pressure_error_is_third_order_in_wave_strength():
    """The Hugoniot osculates the isentrope to second order in the pressure
    jump, so for a weak rarefaction the star pressure differs from the exact
    one at third order: halving the strength divides the error by about 8."""
    errs = []
    for eps in (0.1, 0.05, 0.025):
        p_star, _, _, _, _ = oracle.two_shock([1, 0, 0, 0, 1 + eps], [1, 0, 0, 0, 1.0], GAMMA)
        pe, _ = oracle.riemann_star((1, 0, 1 + eps), (1, 0, 1), GAMMA)
        errs.append(abs(p_star - pe))
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 6.5) & (r < 9.5)), r
    assert errs[0] < 1e-6


def test_two_shock_transonic_fan_state_is_second_order():
    """A pure left rarefaction whose fan straddles x/t = 0: the interpolated
    state differs from the exact fan state (Toro ch. 4 sampling) at second
    order in the wave strength -- halving it divides the density and pressure
    errors by about 4."""
    cL = np.sqrt(GAMMA)
    errs = []
    for eps in (0.1, 0.05, 0.025):
        uL = cL * (1 - eps / 4)
        pR = 1 - eps
        rR = pR ** (1 / GAMMA)
        uR = uL + 2 / (GAMMA - 1) * (cL - np.sqrt(GAMMA * pR / rR))  # left Riemann invariant
        assert uL - cL < 0 < uR - np.sqrt(GAMMA * pR / rR)
        _, _, q, _, _ = oracle.two_shock([1, uL, 0, 0, 1.0], [rR, uR, 0, 0, pR], GAMMA)
        re, ue, pe = oracle.riemann_sample((1, uL, 1), (rR, uR, pR), GAMMA, np.array([0.0]))
        errs.append((abs(q[0] - re[0]), abs(q[4] - pe[0])))
    e = np.array(errs)
    r = e[:-1] / e[1:]
    assert np.all((r > 3.3) & (r < 5.0)), r


@pytest.mark.parametrize("vel", [0.0, 0.3, -0.8, 2.5, -4.0])
def test_two_shock_is_consistent(vel):
    """Equal states: the flux is the Euler flux of that state (supersonic too)."""
    q0 = np.array([0.7, vel, 0.2, -0.4, 1.1])
    p, u, q, F, it = oracle.two_shock(q0, q0, GAMMA)
    E = q0[4] / (GAMMA - 1) + 0.5 * q0[0] * np.sum(q0[1:4] ** 2)
    expect = [q0[0] * vel, q0[0] * vel * vel + q0[4], q0[0] * vel * q0[2], q0[0] * vel * q0[3],
              (E + q0[4]) * vel]
    np.testing.assert_allclose(F, expect, rtol=1e-14, atol=1e-15)
    assert p == q0[4] and u == pytest.approx(vel, abs=1e-15)


def test_two_shock_stationary_and_moving_contacts_are_exact():
    for u in (0.0, 0.6, -0.6):
        L = np.array([2.0, u, 0.1, 0.0, 1.0])
        R = np.array([0.3, u, -0.2, 0.5, 1.0])
        p, us, q, F, _ = oracle.two_shock(L, R, GAMMA)
        assert p == 1.0 and us == pytest.approx(u, abs=1e-15)
        up = L if u >= 0 else R
        np.testing.assert_allclose(q, up, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_two_shock_mirror_symmetry(seed):
    """Reflecting x -> -x swaps the sides and negates the normal velocity; the
    mass, normal-momentum-less and energy fluxes change sign, the normal
    momentum flux does not."""
    rng = np.random.default_rng(seed)
    for _ in range(20):
        L = np.array([rng.uniform(0.1, 3), rng.uniform(-3, 3), rng.normal(), rng.normal(), rng.uniform(0.05, 5)])
        R = np.array([rng.uniform(0.1, 3), rng.uniform(-3, 3), rng.normal(), rng.normal(), rng.uniform(0.05, 5)])
        Lm, Rm = R.copy(), L.copy()
        Lm[1] = -R[1]
        Rm[1] = -L[1]
        _, _, _, F, _ = oracle.two_shock(L, R, GAMMA)
        _, _, _, Fm, _ = oracle.two_shock(Lm, Rm, GAMMA)
        if abs(F[0]) < 1e-9:   # the contact sits on the face: the left-side convention breaks the tie
            continue
        scale = np.abs(F).max() + 1.0
        np.testing.assert_allclose(Fm, [-F[0], F[1], -F[2], -F[3], -F[4]], rtol=0, atol=1e-12 * scale)


# -------------------------------------------------------- whole scheme variants
def run_to(problem, T, limiter, riemann):
    box = oracle.box_of(problem, limiter, riemann)
    Ug = oracle.embed(problem.U)
    t = 0.0
    while t < T * (1 - 1e-14):
        oracle.fill_ghosts(box, Ug)
        dt = min(oracle.compute_dt(box, Ug), T - t)
        rc, _ = oracle.step(box, Ug, dt, nthreads=NT)
        assert rc == 0
        t += dt
    return oracle.interior(Ug)


VARIANTS = [(1, 0), (0, 1), (1, 1)]


@pytest.mark.parametrize("limiter,riemann", VARIANTS)
def test_variant_sod_converges_to_exact_riemann_solution(limiter, riemann):
    T = 0.15
    errs = []
    for n in (32, 64, 128):
        U = run_to(inputs.sod((n, 4, 4)), T, limiter, riemann)
        x = (np.arange(n) + 0.5) / n
        rho_ex, _, _ = oracle.riemann_sample((1, 0, 1), (0.125, 0, 0.1), GAMMA, (x - 0.5) / T)
        errs.append(np.mean(np.abs(U[0, 2, 2, :] - rho_ex)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 4e-3


@pytest.mark.parametrize("limiter,riemann", VARIANTS)
def test_variant_conserves_periodic_density_wave(limiter, riemann):
    pr = inputs.density_wave((12, 10, 8), seed=5)
    U1, _, _, rc = oracle.run(pr, nsteps=8, nthreads=NT, limiter=limiter, riemann=riemann)
    assert rc == 0
    for v in range(5):
        tot0, tot1 = pr.U[v].sum(), U1[v].sum()
        assert abs(tot1 - tot0) <= 1e-12 * np.abs(pr.U[v]).sum()


def _wave_error(n, limiter, T=0.05):
    pr = inputs.density_wave(n, noise=0.0)
    U = run_to(pr, T, limiter, 0)
    x = (np.arange(n) + 0.5) / n
    X = x[None, None, :] + x[None, :, None] + x[:, None, None]
    exact = 1 + 0.1 * np.sin(2 * np.pi * (X - 1.75 * T))
    return np.mean(np.abs(U[0] - exact))


def test_cs_scheme_beats_cw84_on_a_smooth_wave():
    """On a smooth advected wave the CS08 scheme's error is below the CW84
    scheme's at the same resolution (the extrema are not clipped)."""
    for n in (16, 32):
        assert _wave_error(n, 1) < 0.7 * _wave_error(n, 0)


def test_variant_fields_are_validated():
    pr = inputs.uniform((6, 6, 6))
    box = oracle.box_of(pr, 2, 0)
    with pytest.raises(ValueError):
        oracle.compute_dt(box, oracle.embed(pr.U))


# ------------------------------------------- conditioning of the parity cases
def _noise_response(name, variant, samples=2, seed=11):
    from variant_cases import VARIANTS as VV, make_case, scaled_linf
    limiter, riemann = VV[variant] if variant in VV else (0, 0)
    pr = make_case(name)
    Ua, _, _, rc = oracle.run(pr, nsteps=10, nthreads=NT, limiter=limiter, riemann=riemann)
    assert rc == 0
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(samples):
        pn = make_case(name)
        pn.U = pn.U * (1 + rng.integers(-1, 2, pn.U.shape) * 2.0 ** -52)
        Ub, _, _, rc = oracle.run(pn, nsteps=10, nthreads=NT, limiter=limiter, riemann=riemann)
        assert rc == 0
        worst = max(worst, scaled_linf(Ub, Ua))
    return worst


def test_parity_cases_are_as_conditioned_as_claimed():
    """The GPU variant tests assert accumulated ten-step parity only where
    one-ulp input noise moves the oracle's own ten-step result by no more
    than 1e-12; the CS08-sensitive pairs and the Sedov blast move by far more
    (so they are compared one step at a time)."""
    from variant_cases import CS_SENSITIVE, WELL_CONDITIONED
    for name, variant in WELL_CONDITIONED:
        assert _noise_response(name, variant) <= 1e-12, (name, variant)
    for name, variant in CS_SENSITIVE:
        assert _noise_response(name, variant) >= 1e-8, (name, variant)
    assert _noise_response("sedov", "default") >= 1e-3


@pytest.mark.parametrize("variant", ["default", "cs08"])
def test_sedov_l1_response_to_fp32_sized_noise(variant):
    """Relative noise of 2^-24 (FP32 rounding) in the Sedov initial state moves
    the oracle's own 20-step density and energy by up to a few 1e-3 and 1e-2
    in relative L1 (the response varies from one noise sample to the next;
    the largest of three exceeds 1e-3), whatever the limiter: the scale
    against which the mixed-precision CS08 result on this case is judged."""
    from variant_cases import VARIANTS as VV, make_case
    limiter, riemann = VV.get(variant, (0, 0))
    pr = make_case("sedov")
    Ua, _, _, rc = oracle.run(pr, nsteps=20, nthreads=NT, limiter=limiter, riemann=riemann)
    assert rc == 0
    rng = np.random.default_rng(3)
    worst = np.zeros(2)
    for _ in range(3):
        pn = make_case("sedov")
        pn.U = pn.U * (1 + rng.uniform(-1, 1, pn.U.shape) * 2.0 ** -24)
        Ub, _, _, rc = oracle.run(pn, nsteps=20, nthreads=NT, limiter=limiter, riemann=riemann)
        assert rc == 0
        worst = np.maximum(worst, [np.abs(Ub[v] - Ua[v]).sum() / np.abs(Ua[v]).sum() for v in (0, 4)])
    assert np.all(worst > 1e-3), worst
