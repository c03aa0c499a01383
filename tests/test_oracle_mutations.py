"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the oracle's source (a flipped
sign, a swapped operand or index, a dropped term, a wrong constant), builds
it into a temporary library and runs the pin suite against it in a child
process; at least one pin must fail.  The shipped oracle is never touched.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PIN_TESTS = ["tests/test_oracle_ctu.py", "tests/test_oracle_riemann.py", "tests/test_oracle_stages.py",
             "tests/test_oracle_scheme.py", "tests/test_oracle_variants.py"]
VARIANT_PINS_FIRST = PIN_TESTS[4:] + PIN_TESTS[:4]

# (name, file, original text, planted mistake)
MUTANTS = [
    ("ppm interface curvature sign", "hydro_oracle.cpp",
     "- (dm[Z] - dm[Z - s]) / 6.0", "+ (dm[Z] - dm[Z - s]) / 6.0"),
    ("limiter operand swapped", "hydro_oracle.cpp",
     "L = 3.0 * a0 - 2.0 * R;", "L = 3.0 * a0 - 2.0 * L;"),
    ("limited slope without the halving", "hydro_oracle.cpp",
     "double dc = 0.5 * (ap - am);", "double dc = (ap - am);"),
    ("flattening blend operands swapped", "hydro_oracle.cpp",
     "    }\n  }\n  *aL = f * a0 + (1.0 - f) * L;", "    }\n  }\n  *aL = f * L + (1.0 - f) * a0;"),
    ("tracing integral coefficient", "hydro_oracle.cpp",
     "return aR - 0.5 * sig * (dA - (1.0 - 2.0 * sig / 3.0) * a6);",
     "return aR - 0.5 * sig * (dA - (1.0 - sig / 3.0) * a6);"),
    ("left acoustic amplitude sign", "hydro_oracle.cpp",
     "beta[w] = -rho / (2.0 * cs) * du + dp / (2.0 * cs * cs);",
     "beta[w] = rho / (2.0 * cs) * du + dp / (2.0 * cs * cs);"),
    ("entropy amplitude drops the pressure term", "hydro_oracle.cpp",
     "beta[w] = dr - dp / (cs * cs);", "beta[w] = dr;"),
    ("HLLC right bound uses the wrong Roe speed", "hydro_oracle.cpp",
     "SR = fmax(ur + cr, ut + ct);", "SR = fmax(ur + cr, ut - ct);"),
    ("HLLC star energy sign", "hydro_oracle.cpp",
     "(Ss + pl / (rl * (SL - ul)))", "(Ss - pl / (rl * (SL - ul)))"),
    ("transverse correction sign", "hydro_oracle.cpp",
     "val = val - fac[t] * (Fs[t][v * N + Z + s[t]] - Fs[t][v * N + Z]);",
     "val = val + fac[t] * (Fs[t][v * N + Z + s[t]] - Fs[t][v * N + Z]);"),
    ("update reads the wrong face", "hydro_oracle.cpp",
     "val = val - dtdx[d] * (F[Z + G.s[d]] - F[Z]);", "val = val - dtdx[d] * (F[Z] - F[Z - G.s[d]]);"),
    ("flattening shock test on expansions", "hydro_oracle.cpp",
     "un[Z - s] - un[Z + s] > 0.0", "un[Z - s] - un[Z + s] < 0.0"),
    ("reflecting ghosts keep the normal momentum", "hydro_oracle.cpp",
     "if (bc == OB_REFLECT && v == 1 + d) val = -val;", "if (bc == OB_REFLECT && v == 1 + d) val = val;"),
    ("kinetic energy drops a component", "hydro_oracle.cpp",
     "double kin = 0.5 * rho * (u * u + v * v + w * w);", "double kin = 0.5 * rho * (u * u + v * v);"),
    ("exact solver shock function", "exact_riemann.cpp",
     "double root = sqrt(A / (p + B));", "double root = sqrt(A / (p - B));"),
    ("CS08 interface weights", "hydro_oracle.cpp",
     "- 1.0 / 12.0 * (am + a2);", "- 1.0 / 6.0 * (am + a2);"),
    ("CS08 curvature bound constant", "hydro_oracle.cpp",
     "static const double CS_C = 1.25;", "static const double CS_C = 1.0;"),
    ("CS08 parabola curvature factor", "hydro_oracle.cpp",
     "double d2 = 6.0 * (L + R - 2.0 * a0);", "double d2 = 3.0 * (L + R - 2.0 * a0);"),
    ("CS08 interface curvature factor", "hydro_oracle.cpp",
     "double d2 = 3.0 * (a0 - 2.0 * v + a1);", "double d2 = 6.0 * (a0 - 2.0 * v + a1);"),
    ("CS08 extremum test needs both conditions", "hydro_oracle.cpp",
     "if ((R - a0) * (a0 - L) <= 0.0 || (ap - a0) * (a0 - am) <= 0.0) {",
     "if ((R - a0) * (a0 - L) <= 0.0 && (ap - a0) * (a0 - am) <= 0.0) {"),
    ("CS08 edges not scaled", "hydro_oracle.cpp",
     "L = a0 + (L - a0) * (lim / d2);", "L = a0 + (L - a0);"),
    ("two-shock Hugoniot coefficients swapped", "hydro_oracle.cpp",
     "0.5 * (gamma + 1.0) * ps + 0.5 * (gamma - 1.0) * p", "0.5 * (gamma - 1.0) * ps + 0.5 * (gamma + 1.0) * p"),
    ("two-shock star density sign", "hydro_oracle.cpp",
     "1.0 / (1.0 / rk - (ps - pk) / (Wk * Wk))", "1.0 / (1.0 / rk + (ps - pk) / (Wk * Wk))"),
    ("two-shock samples the wrong side", "hydro_oracle.cpp",
     "int left = us >= 0.0;", "int left = us < 0.0;"),
    ("two-shock shock speed frame", "hydro_oracle.cpp",
     "head = tail = Wk / rk - sgn * uk;", "head = tail = Wk / rk + sgn * uk;"),
    ("two-shock fan weights swapped", "hydro_oracle.cpp",
     "q[m] = (1.0 - a) * outer[m] + a * star[m];", "q[m] = a * outer[m] + (1.0 - a) * star[m];"),
    ("two-shock fan tail uses the outer sound speed", "hydro_oracle.cpp",
     "tail = sqrt(gamma * ps / rs) - sgn * us;", "tail = sqrt(gamma * pk / rk) - sgn * us;"),
    ("CTU stage-1 factor 1/2 instead of 1/3", "hydro_oracle.cpp",
     "double fac = dt / (3.0 * b->dx[e]);", "double fac = dt / (2.0 * b->dx[e]);"),
    ("CTU stage-2 factor 1/3 instead of 1/2", "hydro_oracle.cpp",
     "double fac[2] = {dt / (2.0 * b->dx[e]), dt / (2.0 * b->dx[f])};",
     "double fac[2] = {dt / (3.0 * b->dx[e]), dt / (3.0 * b->dx[f])};"),
    ("CTU stage-2 fluxes corrected along the face's own axis", "hydro_oracle.cpp",
     "W_F1 + 5 * pair_index(e, f)) * N,\n                           W + (long)(W_F1 + 5 * pair_index(f, e)) * N};",
     "W_F1 + 5 * pair_index(e, d)) * N,\n                           W + (long)(W_F1 + 5 * pair_index(f, d)) * N};"),
    ("CTU stage-2 pairs swapped", "hydro_oracle.cpp",
     "W_F1 + 5 * pair_index(e, f)) * N,\n                           W + (long)(W_F1 + 5 * pair_index(f, e)) * N};",
     "W_F1 + 5 * pair_index(f, e)) * N,\n                           W + (long)(W_F1 + 5 * pair_index(e, f)) * N};"),
    ("CTU revert rule dropped for p <= 0", "hydro_oracle.cpp",
     "if (!(p > 0.0)) return 0;", "if (!(p > -1e300)) return 0;"),
    ("flattening threshold eps 0.5", "hydro_oracle.cpp",
     "static const double FLAT_EPS = 0.33;", "static const double FLAT_EPS = 0.5;"),
    ("flattening omega1 0.85", "hydro_oracle.cpp",
     "static const double FLAT_OMEGA1 = 0.75;", "static const double FLAT_OMEGA1 = 0.85;"),
    ("flattening omega2 5", "hydro_oracle.cpp",
     "static const double FLAT_OMEGA2 = 10.0;", "static const double FLAT_OMEGA2 = 5.0;"),
    ("flattening tie takes the other neighbour", "hydro_oracle.cpp",
     "long sh = dp1 >= 0.0 ? s : -s;", "long sh = dp1 > 0.0 ? s : -s;"),
    ("tracing reference state is the zone value", "hydro_oracle.cpp",
     "int reaches_fast = side == 0 ? lam[2] > 0.0 : lam[0] < 0.0;", "int reaches_fast = 0;"),
]


def build_mutant(tmp, fname, old, new):
    srcs = []
    for s in ("hydro_oracle.cpp", "exact_riemann.cpp"):
        text = open(os.path.join(ORACLE, s)).read()
        if s == fname:
            assert text.count(old) == 1, f"mutation site not unique in {s}: {old}"
            text = text.replace(old, new)
        dst = os.path.join(tmp, s)
        open(dst, "w").write(text)
        srcs.append(dst)
    lib = os.path.join(tmp, "liboracle_mutant.so")
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", lib] + srcs,
                   check=True)
    return lib


@pytest.mark.parametrize("name,fname,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_planted_mistake(name, fname, old, new):
    with tempfile.TemporaryDirectory() as tmp:
        lib = build_mutant(tmp, fname, old, new)
        env = dict(os.environ, HYDRO_ORACLE_LIB=lib, OMP_WAIT_POLICY="passive")
        # every pin file runs; the planted mistake's own area first, so that -x stops early
        order = VARIANT_PINS_FIRST if name.startswith(("CS08", "two-shock")) else PIN_TESTS
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "-m", "not slow", *order], cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode != 0, f"no pin caught: {name}\n{r.stdout[-2000:]}"
