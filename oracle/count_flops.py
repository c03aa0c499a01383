"""ORACLE TOOLING (test infrastructure only): algorithmic FP64 operation counts.

Builds oracle/flop_count.cpp (the oracle compiled with a counting number
type), runs one step of a seeded input and reports, per stage of the method,
the floating-point operations per unit of work:
  prim     per ghosted zone        dt       per interior zone
  flatten  per extended zone       slopes   per slope-region zone and direction
  trace    per extended zone and direction (interface values, parabolas, tracing)
  riemann  per normal face         ctu1     per once-corrected face (6 pairs)
  ctu2     per final face          update   per interior zone
A flop is one add/sub, mul, div or sqrt; comparisons and min/max are listed
apart.  Run: python -m oracle.count_flops [density_wave|sedov|sod|kelvin_helmholtz]
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

from . import oracle as orc

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(orc.BUILD_DIR, "liboracle_count.so")
STAGES = ("prim", "dt", "flatten", "trace", "riemann", "ctu1", "ctu2", "update", "slopes")
OPS = ("add", "mul", "div", "sqrt", "cmp", "minmax")


def build() -> str:
    src = os.path.join(HERE, "flop_count.cpp")
    deps = [src, os.path.join(HERE, "hydro_oracle.cpp")]
    if os.path.exists(LIB) and all(os.path.getmtime(d) <= os.path.getmtime(LIB) for d in deps):
        return LIB
    os.makedirs(orc.BUILD_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O1", "-ffp-contract=off", "-shared", "-fPIC", "-w", "-o", tmp, src], check=True)
    os.replace(tmp, LIB)
    return LIB


def count(problem) -> dict:
    """{stage: {op: count per unit, 'flops': per unit, 'units': n}} for one step."""
    L = ctypes.CDLL(build())
    D = ctypes.POINTER(ctypes.c_double)
    LL = ctypes.POINTER(ctypes.c_longlong)
    L.oracle_count_step.argtypes = [ctypes.c_int] * 3 + [D, ctypes.c_double, ctypes.c_double,
                                                         ctypes.POINTER(ctypes.c_int), D, ctypes.c_double, LL, LL]
    box = orc.box_of(problem)
    Ug = orc.embed(problem.U)
    orc.fill_ghosts(box, Ug)
    dt = orc.compute_dt(box, Ug)
    dx = np.array(problem.dx, dtype=np.float64)
    bc = (ctypes.c_int * 6)(*[orc.BC_CODES[b] for b in problem.bc])
    out = np.zeros(len(STAGES) * 6, dtype=np.int64)
    units = np.zeros(len(STAGES), dtype=np.int64)
    nx, ny, nz = problem.shape
    rc = L.oracle_count_step(nx, ny, nz, dx.ctypes.data_as(D), problem.gamma, problem.cfl, bc,
                             Ug.ctypes.data_as(D), dt, out.ctypes.data_as(LL), units.ctypes.data_as(LL))
    if rc:
        raise RuntimeError(f"oracle_count_step: {rc}")
    res = {}
    for s, name in enumerate(STAGES):
        per = {op: out[6 * s + k] / units[s] for k, op in enumerate(OPS)}
        per["flops"] = per["add"] + per["mul"] + per["div"] + per["sqrt"]
        per["units"] = int(units[s])
        res[name] = per
    return res


def main(argv):
    from paper_2007_05218_gb300 import inputs
    kind = argv[1] if len(argv) > 1 else "density_wave"
    n = int(argv[2]) if len(argv) > 2 else 32
    make = {"density_wave": lambda: inputs.density_wave(n, seed=0),
            "sedov": lambda: inputs.sedov((n, n, n), seed=0),
            "sod": lambda: inputs.sod((n, n, n)),
            "kelvin_helmholtz": lambda: inputs.kelvin_helmholtz(n, seed=0)}[kind]
    res = count(make())
    print(f"# algorithmic FP64 operations per unit, one step of {kind} {n}^3 (oracle counts)")
    print(f"{'stage':9s} {'unit':22s} " + " ".join(f"{o:>8s}" for o in OPS) + f" {'flops':>9s}")
    unit = {"prim": "ghosted zone", "dt": "interior zone", "flatten": "extended zone",
            "trace": "extended zone x dir", "riemann": "normal face", "ctu1": "corrected face",
            "ctu2": "final face", "update": "interior zone", "slopes": "slope zone x dir"}
    for s in STAGES:
        r = res[s]
        print(f"{s:9s} {unit[s]:22s} " + " ".join(f"{r[o]:8.2f}" for o in OPS) + f" {r['flops']:9.2f}")
    total = sum(res[s]["flops"] * res[s]["units"] for s in STAGES if s != "dt") / res["update"]["units"]
    print(f"total flops per interior zone-update at {n}^3 (extended regions included, dt reduction"
          f" counted inside prim on the GPU so excluded here): {total:.1f}")


if __name__ == "__main__":
    main(sys.argv)
