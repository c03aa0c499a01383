"""Pins of the oracle's exact Riemann solver (CPU only).

The exact solver is itself a pin for the whole scheme (Sod tests), so it is
checked against values printed in a textbook table and against the jump and
invariant relations any exact solution must satisfy.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toro_riemann_star.txt")
GAMMA = 1.4


def _rows():
    return np.loadtxt(GOLDEN, comments="#")


@pytest.mark.parametrize("row", range(5))
def test_star_state_matches_textbook_table(row):
    r = _rows()[row]
    L, R = tuple(r[0:3]), tuple(r[3:6])
    ps, us = oracle.riemann_star(L, R, GAMMA)
    eps = 1e-9 * max(1.0, abs(us))
    rl, _, _ = oracle.riemann_sample(L, R, GAMMA, [us - eps])
    rr, _, _ = oracle.riemann_sample(L, R, GAMMA, [us + eps])
    # the table prints ~6 significant digits of values computed from rounded inputs
    assert ps == pytest.approx(r[6], rel=2e-5, abs=6e-6)
    assert us == pytest.approx(r[7], rel=2e-5, abs=6e-6)
    assert rl[0] == pytest.approx(r[8], rel=2e-5, abs=6e-6)
    assert rr[0] == pytest.approx(r[9], rel=2e-5, abs=6e-6)


def _shock_jump_residuals(pre, post, S):
    """Rankine-Hugoniot residuals (mass, momentum, energy) across a shock of speed S."""
    (r0, u0, p0), (r1, u1, p1) = pre, post
    E0 = p0 / (GAMMA - 1) + 0.5 * r0 * u0 * u0
    E1 = p1 / (GAMMA - 1) + 0.5 * r1 * u1 * u1
    U0 = np.array([r0, r0 * u0, E0])
    U1 = np.array([r1, r1 * u1, E1])
    F0 = np.array([r0 * u0, r0 * u0 * u0 + p0, (E0 + p0) * u0])
    F1 = np.array([r1 * u1, r1 * u1 * u1 + p1, (E1 + p1) * u1])
    return (F1 - F0) - S * (U1 - U0)


def test_sod_right_shock_satisfies_rankine_hugoniot():
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = oracle.riemann_star(L, R, GAMMA)
    # locate the right shock by sampling: the last S where the state differs from R
    S = np.linspace(us + 1e-6, 3.0, 200001)
    rho, u, p = oracle.riemann_sample(L, R, GAMMA, S)
    i = np.nonzero(rho != R[0])[0].max()
    shock_speed = 0.5 * (S[i] + S[i + 1])
    post = (rho[i], u[i], p[i])
    res = _shock_jump_residuals(R, post, shock_speed)
    scale = np.array([1.0, 1.0, 2.5])
    assert np.all(np.abs(res) / scale < 5e-5)
    assert post[1] == pytest.approx(us, rel=1e-12)
    assert post[2] == pytest.approx(ps, rel=1e-12)


def test_sod_left_rarefaction_keeps_riemann_invariant_and_entropy():
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = oracle.riemann_star(L, R, GAMMA)
    cL = np.sqrt(GAMMA * L[2] / L[0])
    cs = cL * (ps / L[2]) ** ((GAMMA - 1) / (2 * GAMMA))
    S = np.linspace(-cL + 1e-9, us - cs - 1e-9, 101)  # inside the fan
    rho, u, p = oracle.riemann_sample(L, R, GAMMA, S)
    c = np.sqrt(GAMMA * p / rho)
    J = u + 2 * c / (GAMMA - 1)
    np.testing.assert_allclose(J, 2 * cL / (GAMMA - 1), rtol=1e-12)
    np.testing.assert_allclose(p / rho ** GAMMA, L[2] / L[0] ** GAMMA, rtol=1e-12)
    # self-similar: the fan's characteristic u - c equals x/t
    np.testing.assert_allclose(u - c, S, atol=1e-12)


def test_two_rarefaction_closed_form():
    """When both waves are rarefactions p* has a closed form (two-rarefaction solution)."""
    L, R = (1.0, -2.0, 0.4), (1.0, 2.0, 0.4)
    ps, us = oracle.riemann_star(L, R, GAMMA)
    cl = np.sqrt(GAMMA * L[2] / L[0])
    cr = np.sqrt(GAMMA * R[2] / R[0])
    z = (GAMMA - 1) / (2 * GAMMA)
    num = cl + cr - 0.5 * (GAMMA - 1) * (R[1] - L[1])
    den = cl / L[2] ** z + cr / R[2] ** z
    assert ps == pytest.approx((num / den) ** (1 / z), rel=1e-12)
    assert us == pytest.approx(0.0, abs=1e-14)


def test_trivial_problem_returns_the_state():
    ps, us = oracle.riemann_star((0.7, 0.3, 2.0), (0.7, 0.3, 2.0), GAMMA)
    assert ps == pytest.approx(2.0, rel=1e-14)
    assert us == pytest.approx(0.3, rel=1e-14)
