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
PIN_TESTS = ["tests/test_oracle_riemann.py", "tests/test_oracle_stages.py", "tests/test_oracle_scheme.py"]

# (name, file, original text, planted mistake)
MUTANTS = [
    ("ppm interface curvature sign", "hydro_oracle.cpp",
     "- (dm[Z] - dm[Z - s]) / 6.0", "+ (dm[Z] - dm[Z - s]) / 6.0"),
    ("limiter operand swapped", "hydro_oracle.cpp",
     "L = 3.0 * a0 - 2.0 * R;", "L = 3.0 * a0 - 2.0 * L;"),
    ("limited slope without the halving", "hydro_oracle.cpp",
     "double dc = 0.5 * (ap - am);", "double dc = (ap - am);"),
    ("flattening blend operands swapped", "hydro_oracle.cpp",
     "*aL = f * a0 + (1.0 - f) * L;", "*aL = f * L + (1.0 - f) * a0;"),
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
        env = dict(os.environ, HYDRO_ORACLE_LIB=lib)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "-m", "not slow", *PIN_TESTS], cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode != 0, f"no pin caught: {name}\n{r.stdout[-2000:]}"
