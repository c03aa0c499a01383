"""Stage-level pins of the oracle (CPU only): each stage against a closed form,
an invariant or a library routine, chosen so that a dropped term, a wrong sign
or a swapped index in that stage fails a test here."""
import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import inputs

GAMMA = 1.4
rng = np.random.default_rng(12345)


def euler_flux(d, q, gamma):
    """Physical Euler flux normal to axis d of primitive q = (rho, u, v, w, p)."""
    rho, vel, p = q[0], np.asarray(q[1:4]), q[4]
    E = p / (gamma - 1) + 0.5 * rho * vel @ vel
    F = np.empty(5)
    F[0] = rho * vel[d]
    F[1:4] = rho * vel[d] * vel
    F[1 + d] += p
    F[4] = (E + p) * vel[d]
    return F


def random_state():
    return np.array([rng.uniform(0.2, 3.0), *rng.uniform(-1.5, 1.5, 3), rng.uniform(0.1, 5.0)])


# ----------------------------------------------------------------- HLLC
@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_consistency_equal_states_give_physical_flux(d):
    for _ in range(50):
        q = random_state()
        F = oracle.hllc(d, q, q, GAMMA)
        np.testing.assert_allclose(F, euler_flux(d, q, GAMMA), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_supersonic_is_upwind_flux(d):
    for _ in range(20):
        qL, qR = random_state(), random_state()
        cL = np.sqrt(GAMMA * qL[4] / qL[0])
        cR = np.sqrt(GAMMA * qR[4] / qR[0])
        qL[1 + d] = 3.0 * max(cL, cR) + 1.0
        qR[1 + d] = 3.0 * max(cL, cR) + 1.0
        np.testing.assert_allclose(oracle.hllc(d, qL, qR, GAMMA), euler_flux(d, qL, GAMMA), rtol=1e-14)
        qL[1 + d] *= -1.0
        qR[1 + d] *= -1.0
        np.testing.assert_allclose(oracle.hllc(d, qL, qR, GAMMA), euler_flux(d, qR, GAMMA), rtol=1e-14)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_resolves_stationary_contact_exactly(d):
    qL = np.array([1.0, 0, 0, 0, 2.0])
    qR = np.array([0.1, 0, 0, 0, 2.0])
    t = [a for a in range(3) if a != d]
    qL[1 + t[0]] = 0.3  # transverse shear is carried by the contact too
    qR[1 + t[1]] = -0.7
    F = oracle.hllc(d, qL, qR, GAMMA)
    expect = np.zeros(5)
    expect[1 + d] = 2.0
    np.testing.assert_array_equal(F, expect)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_mirror_symmetry(d):
    for _ in range(20):
        qL, qR = random_state(), random_state()
        F = oracle.hllc(d, qL, qR, GAMMA)
        mL, mR = qR.copy(), qL.copy()
        mL[1 + d] *= -1
        mR[1 + d] *= -1
        Fm = oracle.hllc(d, mL, mR, GAMMA)
        sign = -np.ones(5)
        sign[1 + d] = 1.0
        np.testing.assert_allclose(Fm, sign * F, rtol=1e-12, atol=1e-13)


def test_hllc_is_exact_for_a_stationary_shock():
    """Rankine-Hugoniot-related states with zero shock speed: F_L = F_R must come out."""
    g = GAMMA
    M = 2.5
    rho1, p1 = 1.0, 1.0
    u1 = M * np.sqrt(g * p1 / rho1)
    rho2 = rho1 * (g + 1) * M * M / ((g - 1) * M * M + 2)
    p2 = p1 * (2 * g * M * M - (g - 1)) / (g + 1)
    u2 = rho1 * u1 / rho2
    qL = np.array([rho1, u1, 0, 0, p1])
    qR = np.array([rho2, u2, 0, 0, p2])
    FL, FR = euler_flux(0, qL, g), euler_flux(0, qR, g)
    np.testing.assert_allclose(FL, FR, rtol=1e-13)
    np.testing.assert_allclose(oracle.hllc(0, qL, qR, g), FL, rtol=1e-12)


# ------------------------------------------------------------------ PPM
def test_limited_slope_values():
    assert oracle.limited_slope(0.0, 1.0, 2.0) == 1.0
    assert oracle.limited_slope(2.0, 1.0, 0.0) == -1.0
    assert oracle.limited_slope(0.0, 0.1, 2.0) == pytest.approx(0.2)
    assert oracle.limited_slope(0.0, 1.0, 1.0) == 0.0
    assert oracle.limited_slope(0.0, 1.0, 0.5) == 0.0


def test_ppm_reproduces_linear_data_exactly():
    a = 2.0 + 0.25 * np.arange(20)
    aL, aR = oracle.ppm_line(a)
    s = slice(2, 18)
    np.testing.assert_allclose(aL[s], a[s] - 0.125, rtol=0, atol=1e-14)
    np.testing.assert_allclose(aR[s], a[s] + 0.125, rtol=0, atol=1e-14)
    a6 = 6 * (a[s] - 0.5 * (aL[s] + aR[s]))
    assert np.max(np.abs(a6)) < 1e-13


def test_ppm_interface_values_exact_for_cubic_cell_averages():
    """Unlimited 4th-order interface formula is exact for cell averages of a cubic."""
    h = 0.01
    xe = 1.0 + h * np.arange(31)
    prim = lambda x: x ** 4 / 4 + x * x  # antiderivative of f = x^3 + 2x
    f = lambda x: x ** 3 + 2 * x
    avg = (prim(xe[1:]) - prim(xe[:-1])) / h
    aL, aR = oracle.ppm_line(avg)
    s = slice(2, 28)
    np.testing.assert_allclose(aR[s], f(xe[1:][s]), rtol=2e-12)
    np.testing.assert_allclose(aL[s], f(xe[:-1][s]), rtol=2e-12)


def test_ppm_limiter_creates_no_new_extrema():
    for trial in range(20):
        a = rng.normal(size=60).cumsum() if trial % 2 else rng.uniform(-1, 1, 60)
        aL, aR = oracle.ppm_line(a)
        i = np.arange(2, 58)
        tol = 1e-13
        assert np.all(aL[i] >= np.minimum(a[i - 1], a[i]) - tol)
        assert np.all(aL[i] <= np.maximum(a[i - 1], a[i]) + tol)
        assert np.all(aR[i] >= np.minimum(a[i], a[i + 1]) - tol)
        assert np.all(aR[i] <= np.maximum(a[i], a[i + 1]) + tol)
        assert np.all((aR[i] - a[i]) * (a[i] - aL[i]) >= -tol)
        a6 = 6 * (a[i] - 0.5 * (aL[i] + aR[i]))
        assert np.all(np.abs(a6) <= np.abs(aR[i] - aL[i]) + tol)


def test_ppm_full_flattening_gives_first_order():
    a = rng.uniform(0, 1, 30)
    aL, aR = oracle.ppm_line(a, np.ones(30))
    np.testing.assert_array_equal(aL[2:28], a[2:28])
    np.testing.assert_array_equal(aR[2:28], a[2:28])


# ------------------------------------------------------------ flattening
def test_flattening_zero_on_smooth_data_and_one_at_strong_shock():
    x = np.linspace(0, 1, 40)
    f = oracle.flatten_line(1.0 + 0.1 * np.sin(2 * np.pi * x), 0.2 * np.cos(2 * np.pi * x))
    assert np.all(f[3:37] == 0.0)
    p = np.where(np.arange(20) < 10, 10.0, 1.0)  # compressive: u drops across the jump
    u = np.where(np.arange(20) < 10, 1.0, 0.0)
    f = oracle.flatten_line(p, u)
    assert f[9] == 1.0 and f[10] == 1.0
    assert f[5] == 0.0 and f[15] == 0.0
    f = oracle.flatten_line(p, -u)  # expansion: no flattening
    assert np.all(f[3:17] == 0.0)


# --------------------------------------------------------------- tracing
def _line(n=24, subsonic=True):
    x = np.linspace(0, 1, n)
    q = np.empty((5, n))
    q[0] = 1.0 + 0.2 * np.sin(5 * x)
    q[1] = 0.3 * np.cos(3 * x) if subsonic else 4.0 + 0.1 * x
    q[2] = 0.1 * x
    q[3] = -0.2 * x * x
    q[4] = 1.0 + 0.1 * np.cos(4 * x)
    c = np.sqrt(GAMMA * q[4] / q[0])
    return q, c


def test_tracing_with_zero_dt_returns_the_limited_edge_values():
    q, c = _line()
    chi = np.zeros(q.shape[1])
    qm, qp = oracle.trace_line(q, c, chi, 0.0)
    for m in range(5):
        aL, aR = oracle.ppm_line(q[m], chi)
        np.testing.assert_array_equal(qm[m, 2:-2], aL[2:-2])
        np.testing.assert_array_equal(qp[m, 2:-2], aR[2:-2])


def test_tracing_uniform_line_is_identity():
    q = np.tile(np.array([[1.3], [0.4], [-0.2], [0.1], [0.8]]), (1, 16))
    c = np.sqrt(GAMMA * q[4] / q[0])
    qm, qp = oracle.trace_line(q, c, np.zeros(16), 0.3)
    np.testing.assert_array_equal(qm[:, 2:-2], q[:, 2:-2])
    np.testing.assert_array_equal(qp[:, 2:-2], q[:, 2:-2])


def test_tracing_supersonic_left_edge_is_zone_value():
    q, c = _line(subsonic=False)
    qm, qp = oracle.trace_line(q, c, np.zeros(q.shape[1]), 0.05)
    np.testing.assert_array_equal(qm[:, 2:-2], q[:, 2:-2])


def test_tracing_pure_entropy_wave_is_parabola_average_over_upwind_domain():
    """With uniform u, p only the entropy wave carries information: the right-edge
    density must be the mean of the zone parabola over [1 - sigma, 1] (sigma = u dt/dx),
    computed here by Gauss-Legendre quadrature of the parabola."""
    n = 24
    x = np.linspace(0, 1, n)
    q = np.empty((5, n))
    q[0] = 1.0 + 0.3 * np.sin(4 * x)
    q[1], q[2], q[3], q[4] = 0.4, 0.0, 0.0, 1.0
    c = np.sqrt(GAMMA * q[4] / q[0])
    dtdx = 0.6
    qm, qp = oracle.trace_line(q, c, np.zeros(n), dtdx)
    aL, aR = oracle.ppm_line(q[0])
    sig = 0.4 * dtdx
    xg, wg = np.polynomial.legendre.leggauss(4)
    for i in range(2, n - 2):
        a6 = 6 * (q[0, i] - 0.5 * (aL[i] + aR[i]))
        par = lambda xi: aL[i] + xi * (aR[i] - aL[i] + a6 * (1 - xi))
        xi = 1 - sig + 0.5 * sig * (xg + 1)
        mean = 0.5 * np.sum(wg * par(xi))
        assert qp[0, i] == pytest.approx(mean, rel=1e-13)
        assert qp[4, i] == pytest.approx(1.0, rel=1e-14)
        assert qp[1, i] == pytest.approx(0.4, rel=1e-13)


# ------------------------------------------------- cons<->prim, ghosts, dt
def test_cons_prim_round_trip():
    pr = inputs.kelvin_helmholtz(8, seed=3)
    box = oracle.box_of(pr)
    Ug = oracle.embed(pr.U)
    q, c = oracle.prim(box, Ug)
    qi = oracle.interior(q)
    U = pr.U
    np.testing.assert_allclose(qi[0], U[0], rtol=0)
    for a in range(3):
        np.testing.assert_allclose(qi[1 + a] * qi[0], U[1 + a], rtol=1e-15, atol=1e-17)
    np.testing.assert_allclose(qi[4], 2.5, rtol=4e-15)
    np.testing.assert_allclose(oracle.interior(c[None])[0], np.sqrt(1.4 * 2.5 / U[0]), rtol=1e-15)


@pytest.mark.parametrize("bc,mode", [("periodic", "wrap"), ("outflow", "edge"), ("reflect", "symmetric")])
def test_ghost_fill_matches_numpy_padding(bc, mode):
    U = rng.uniform(0.5, 1.5, (5, 6, 5, 7))
    box = oracle.make_box((7, 5, 6), (0.1, 0.1, 0.1), GAMMA, 0.5, (bc,) * 6)
    Ug = oracle.embed(U)
    oracle.fill_ghosts(box, Ug)
    for v in range(5):
        ref = np.pad(U[v], 4, mode=mode)
        if bc == "reflect" and v in (1, 2, 3):
            # the normal momentum flips sign in the ghosts normal to its axis
            axis = 2 - (v - 1)
            sl = [slice(None)] * 3
            for side in (slice(0, 4), slice(-4, None)):
                sl[axis] = side
                ref[tuple(sl)] *= -1
        np.testing.assert_array_equal(Ug[v], ref)


def test_dt_closed_form_on_uniform_state():
    pr = inputs.uniform(8, rho=1.3, vel=(0.3, -0.9, 0.1), p=0.7, gamma=GAMMA)
    pr.dx = (0.1, 0.05, 0.2)
    box = oracle.box_of(pr)
    dt = oracle.compute_dt(box, oracle.embed(pr.U))
    c = np.sqrt(GAMMA * 0.7 / 1.3)
    expect = 0.5 * min(0.1 / (0.3 + c), 0.05 / (0.9 + c), 0.2 / (0.1 + c))
    assert dt == pytest.approx(expect, rel=1e-14)


def _parabola_mean(aL, aR, a0, lo, hi):
    """Mean of the zone parabola over [lo, hi] of the zone's unit interval (quadrature)."""
    a6 = 6 * (a0 - 0.5 * (aL + aR))
    xg, wg = np.polynomial.legendre.leggauss(4)
    xi = lo + 0.5 * (hi - lo) * (xg + 1)
    return 0.5 * np.sum(wg * (aL + xi * (aR - aL + a6 * (1 - xi))))


@pytest.mark.parametrize("u0", [2.2, 0.4, -0.4, -2.2])
def test_tracing_projects_each_characteristic_on_its_own_upwind_average(u0):
    """Characteristic tracing: with the zone-centred left eigenvectors
    l- = (0, -rho/2c, 1/2c^2), l0 = (1, 0, -1/c^2), l+ = (0, rho/2c, 1/2c^2) in
    (rho, u_n, p), each wave that reaches an edge carries its own upwind average
    of the parabolas to it, l.q_edge = l.I(sigma_wave), and a wave that does
    not reach leaves l.q_edge = l.q_ref.  Sub- and supersonic, both directions."""
    n = 24
    x = np.linspace(0, 1, n)
    q = np.empty((5, n))
    q[0] = 1.0 + 0.2 * np.sin(5 * x)
    q[1] = u0 + 0.1 * np.cos(3 * x)
    q[2] = 0.1 * np.sin(2 * x)
    q[3] = -0.2 * x * x
    q[4] = 1.0 + 0.1 * np.cos(4 * x)
    c = np.sqrt(GAMMA * q[4] / q[0])
    dtdx = 0.15
    qm, qp = oracle.trace_line(q, c, np.zeros(n), dtdx)
    par = [oracle.ppm_line(q[m]) for m in range(5)]
    for i in range(3, n - 3):
        rho, u, cs = q[0, i], q[1, i], c[i]
        lvec = {-1: np.array([0.0, -rho / (2 * cs), 1 / (2 * cs * cs)]),
                0: np.array([1.0, 0.0, -1 / (cs * cs)]),
                1: np.array([0.0, rho / (2 * cs), 1 / (2 * cs * cs)])}
        lam = {-1: u - cs, 0: u, 1: u + cs}
        for side, qe in ((0, qp), (1, qm)):
            def avg(m, sig):
                aL, aR = par[m][0][i], par[m][1][i]
                return (_parabola_mean(aL, aR, q[m, i], 1 - sig, 1) if side == 0
                        else _parabola_mean(aL, aR, q[m, i], 0, sig))
            reaches = (lambda l: l > 0) if side == 0 else (lambda l: l < 0)
            fast = 1 if side == 0 else -1
            ref = ([avg(m, abs(lam[fast]) * dtdx) for m in range(5)] if reaches(lam[fast])
                   else list(q[:, i]))
            edge = np.array([qe[0, i], qe[1, i], qe[4, i]])
            for nu in (-1, 0, 1):
                if reaches(lam[nu]):
                    sig = abs(lam[nu]) * dtdx
                    target = np.array([avg(0, sig), avg(1, sig), avg(4, sig)])
                else:
                    target = np.array([ref[0], ref[1], ref[4]])
                assert lvec[nu] @ edge == pytest.approx(lvec[nu] @ target, rel=1e-11, abs=1e-12), (i, side, nu)
            for m in (2, 3):  # transverse velocities ride the entropy wave
                expect = avg(m, abs(u) * dtdx) if reaches(lam[0]) else ref[m]
                assert qe[m, i] == pytest.approx(expect, rel=1e-11, abs=1e-13)
