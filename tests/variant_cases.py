"""Inputs of the method-variant parity tests (seeded, synthetic; no method
arithmetic here).

Conditioning decides how a case can be compared.  Ten steps of the oracle
from an initial state perturbed by one ulp move the result (relative
L-infinity, momenta scaled by the largest momentum) by about 2e-15 on the
WELL_CONDITIONED pairs below.  They move it by 2e-5 to 1e-4 under the CS08
limiter on the colliding-flow and density-wave cases: its sign tests on
second differences flip where symmetry makes a second difference zero up to
rounding.  On the Sedov blast they move it by 5e-2 for every method, since
the pressure behind the front is a small difference of large energies.
Accumulated ten-step parity is only asserted on well-conditioned pairs; every
pair is also compared one step at a time from the oracle's own state
(tests/test_gpu_variants.py), and tests/test_oracle_variants.py pins the
conditioning claims.
"""
import numpy as np

from paper_2007_05218_gb300 import hydro, inputs

CS, TS = hydro.HYDRO_LIMITER_CS08, hydro.HYDRO_RIEMANN_TWO_SHOCK
VARIANTS = {"cs08": (CS, 0), "two_shock": (0, TS), "cs08_two_shock": (CS, TS)}


def colliding(pr):
    """Two streams meeting at the x midplane at +-2 (both waves shocks)."""
    nx = pr.shape[0]
    U = pr.U.copy()
    rho = U[0]
    u = np.where(np.arange(nx)[None, None, :] < nx // 2, 2.0, -2.0) * np.ones_like(rho)
    U[4] = U[4] - 0.5 * U[1] ** 2 / rho + 0.5 * rho * u * u
    U[1] = rho * u
    pr.U = U
    return pr


CASES = {
    "sod_x": lambda: inputs.sod((32, 6, 5), axis=0),
    "sod_z_mirror": lambda: inputs.sod((6, 5, 20), axis=2, flip=True),
    "density_wave_ragged": lambda: inputs.density_wave((20, 12, 9), seed=3),
    "sedov": lambda: inputs.sedov((17, 16, 18), seed=2),
    "kelvin_helmholtz_reflect_y": lambda: inputs.kelvin_helmholtz((12, 16, 10), seed=4),
    "colliding_flows": lambda: colliding(inputs.uniform((16, 5, 6), vel=(0.0, 0.0, 0.0), bc="reflect")),
}

WELL_CONDITIONED = sorted(
    [(name, v) for name in ("sod_x", "sod_z_mirror", "kelvin_helmholtz_reflect_y") for v in VARIANTS]
    + [(name, "two_shock") for name in ("density_wave_ragged", "colliding_flows")])
CS_SENSITIVE = [(name, v) for name in ("density_wave_ragged", "colliding_flows") for v in ("cs08", "cs08_two_shock")]


def make_case(name):
    return CASES[name]()


def scaled_linf(a, b):
    """max over fields of max|a - b| / scale, with density and energy scaled
    by their own maxima and the momenta by the largest momentum component."""
    mom = max(np.max(np.abs(b[v])) for v in (1, 2, 3))
    sc = [np.max(np.abs(b[0])), mom, mom, mom, np.max(np.abs(b[4]))]
    return max(np.max(np.abs(a[v] - b[v])) / (sc[v] if sc[v] > 0 else 1.0) for v in range(5))
