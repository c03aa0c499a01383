"""ctypes wrapper of the oracle (test infrastructure only).

Arrays crossing into C are float64, C-contiguous, laid out [field][k][j][i]
over the ghosted box (no padding).  `embed`/`interior` convert between the
interior-only arrays built by the input generators and that layout.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = ("hydro_oracle.cpp", "exact_riemann.cpp")
NG = 4
BC_CODES = {"periodic": 0, "outflow": 1, "reflect": 2}

# intermediate field offsets (in fields of Ng doubles) inside the step dump
W_Q, W_C, W_CHI, W_QM, W_QP, W_F0, W_F1, W_F, W_NFIELDS = 0, 5, 6, 7, 22, 37, 52, 82, 97
PAIRS = ((0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1))


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no fused multiply-add, OpenMP over k-planes)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    if not force and os.path.exists(LIB_PATH):
        mt = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(s) <= mt for s in srcs):
            return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
           "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class ObBox(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("ng", ctypes.c_int), ("dx", ctypes.c_double * 3), ("gamma", ctypes.c_double),
                ("cfl", ctypes.c_double), ("bc", ctypes.c_int * 6), ("limiter", ctypes.c_int),
                ("riemann", ctypes.c_int)]

# method variants: CW84 limiter (0) or Colella-Sekora (1); HLLC (0) or two-shock (1)
LIMITER_CW84, LIMITER_CS08 = 0, 1
RIEMANN_HLLC, RIEMANN_TWO_SHOCK = 0, 1


_lib = None
_lock = threading.Lock()
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    """The oracle library; HYDRO_ORACLE_LIB may name another build of it (the
    mutation tests load deliberately broken copies that way)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("HYDRO_ORACLE_LIB")
            if not path:
                build()
                path = LIB_PATH
            L = ctypes.CDLL(path)
            P = ctypes.POINTER(ObBox)
            L.oracle_fill_ghosts.argtypes = [P, _D]
            L.oracle_compute_dt.argtypes = [P, _D, _D]
            L.oracle_prim.argtypes = [P, _D, _D, _D]
            L.oracle_step.argtypes = [P, _D, ctypes.c_double, _D, ctypes.c_int]
            L.oracle_run.argtypes = [P, _D, ctypes.c_int, _D, _D, ctypes.c_int]
            L.oracle_hllc.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, _D]
            L.oracle_ppm_line.argtypes = [_D, _D, ctypes.c_int, _D, _D]
            L.oracle_limited_slope.argtypes = [ctypes.c_double] * 3
            L.oracle_limited_slope.restype = ctypes.c_double
            L.oracle_trace_line.argtypes = [_D, _D, _D, ctypes.c_int, ctypes.c_double, _D, _D]
            L.oracle_flatten_line.argtypes = [_D, _D, ctypes.c_int, _D]
            L.oracle_ppm_line_cs.argtypes = [_D, _D, ctypes.c_int, _D, _D]
            L.oracle_two_shock.argtypes = [_D, _D, ctypes.c_double, _D, _D, _D]
            L.oracle_riemann_star.argtypes = [ctypes.c_double] * 7 + [_D, _D]
            L.oracle_riemann_sample.argtypes = [ctypes.c_double] * 7 + [_D, ctypes.c_int, _D, _D, _D]
            L.oracle_branch_hits.argtypes = [ctypes.POINTER(ctypes.c_long), ctypes.c_int, ctypes.c_int]
            L.oracle_set_wall_r11.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def make_box(shape, dx, gamma, cfl, bc, ng: int = NG, limiter: int = 0, riemann: int = 0) -> ObBox:
    """shape = (nx, ny, nz); bc = six names (xlo, xhi, ylo, yhi, zlo, zhi)."""
    b = ObBox()
    b.nx, b.ny, b.nz = (int(v) for v in shape)
    b.ng = ng
    for a in range(3):
        b.dx[a] = float(dx[a])
    b.gamma = float(gamma)
    b.cfl = float(cfl)
    for a in range(6):
        b.bc[a] = BC_CODES[bc[a]]
    b.limiter = int(limiter)
    b.riemann = int(riemann)
    return b


def box_of(problem, limiter: int = 0, riemann: int = 0) -> ObBox:
    return make_box(problem.shape, problem.dx, problem.gamma, problem.cfl, problem.bc,
                    limiter=limiter, riemann=riemann)


def embed(U: np.ndarray, ng: int = NG) -> np.ndarray:
    """[v][nz][ny][nx] interior -> [v][nz+2g][ny+2g][nx+2g] with zero ghosts."""
    nv, nz, ny, nx = U.shape
    out = np.zeros((nv, nz + 2 * ng, ny + 2 * ng, nx + 2 * ng))
    out[:, ng:ng + nz, ng:ng + ny, ng:ng + nx] = U
    return out


def interior(Ug: np.ndarray, ng: int = NG) -> np.ndarray:
    return np.ascontiguousarray(Ug[:, ng:-ng, ng:-ng, ng:-ng])


def fill_ghosts(box: ObBox, Ug: np.ndarray) -> None:
    rc = lib().oracle_fill_ghosts(ctypes.byref(box), _p(Ug))
    if rc:
        raise ValueError(f"oracle_fill_ghosts: {rc}")


def compute_dt(box: ObBox, Ug: np.ndarray) -> float:
    dt = ctypes.c_double()
    rc = lib().oracle_compute_dt(ctypes.byref(box), _p(Ug), ctypes.byref(dt))
    if rc:
        raise ValueError(f"oracle_compute_dt: {rc}")
    return dt.value


def prim(box: ObBox, Ug: np.ndarray):
    n = Ug[0].size
    q = np.zeros((5,) + Ug.shape[1:])
    c = np.zeros(Ug.shape[1:])
    lib().oracle_prim(ctypes.byref(box), _p(Ug), _p(q), _p(c))
    return q, c


def step(box: ObBox, Ug: np.ndarray, dt: float, dump: bool = False, nthreads: int = 1):
    """One update of the ghost-filled state Ug in place.  Returns (status, dump-or-None)."""
    W = np.zeros((W_NFIELDS,) + Ug.shape[1:]) if dump else None
    rc = lib().oracle_step(ctypes.byref(box), _p(Ug), float(dt),
                           _p(W) if dump else ctypes.cast(None, _D), int(nthreads))
    if rc == -1:
        raise ValueError("oracle_step: invalid box")
    return rc, W


def run(problem, nsteps: int | None = None, nthreads: int = 1, limiter: int = 0, riemann: int = 0):
    """Advance `problem` nsteps (default problem.nsteps) with dt from the state,
    with the given limiter and Riemann solver.

    Returns (U_interior, t, dts, status).
    """
    n = problem.nsteps if nsteps is None else int(nsteps)
    box = box_of(problem, limiter, riemann)
    Ug = embed(problem.U)
    dts = np.zeros(max(n, 1))
    t = ctypes.c_double()
    rc = lib().oracle_run(ctypes.byref(box), _p(Ug), n, _p(dts), ctypes.byref(t), int(nthreads))
    if rc == -1:
        raise ValueError("oracle_run: invalid box")
    return interior(Ug), t.value, dts[:n], rc


def hllc(d: int, qL, qR, gamma: float) -> np.ndarray:
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    F = np.zeros(5)
    lib().oracle_hllc(int(d), _p(qL), _p(qR), float(gamma), _p(F))
    return F


def ppm_line(a, chi=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    chi = np.zeros_like(a) if chi is None else np.ascontiguousarray(chi, dtype=np.float64)
    aL = np.full_like(a, np.nan)
    aR = np.full_like(a, np.nan)
    lib().oracle_ppm_line(_p(a), _p(chi), a.size, _p(aL), _p(aR))
    return aL, aR


def ppm_line_cs(a, chi=None):
    """Colella-Sekora parabolas of a 1D line; zones 2..n-3 are written."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    chi = np.zeros_like(a) if chi is None else np.ascontiguousarray(chi, dtype=np.float64)
    aL = np.full_like(a, np.nan)
    aR = np.full_like(a, np.nan)
    lib().oracle_ppm_line_cs(_p(a), _p(chi), a.size, _p(aL), _p(aR))
    return aL, aR


def two_shock(L, R, gamma: float):
    """Two-shock solver on normal-frame states (rho, u_n, u_t1, u_t2, p).
    Returns (p*, u*, interface state q[5], flux F[5], Newton steps)."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    pu, q, F = np.zeros(2), np.zeros(5), np.zeros(5)
    it = lib().oracle_two_shock(_p(L), _p(R), float(gamma), _p(pu), _p(q), _p(F))
    return pu[0], pu[1], q, F, it


def limited_slope(am: float, a0: float, ap: float) -> float:
    return lib().oracle_limited_slope(float(am), float(a0), float(ap))


def trace_line(q, c, chi, dtdx: float):
    """q: [5][n] normal-frame primitive (rho, u_n, u_t1, u_t2, p)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = q.shape[1]
    c = np.ascontiguousarray(c, dtype=np.float64)
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    qm = np.full_like(q, np.nan)
    qp = np.full_like(q, np.nan)
    lib().oracle_trace_line(_p(q), _p(c), _p(chi), n, float(dtdx), _p(qm), _p(qp))
    return qm, qp


def flatten_line(p, u):
    p = np.ascontiguousarray(p, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.full_like(p, np.nan)
    lib().oracle_flatten_line(_p(p), _p(u), p.size, _p(f))
    return f


def riemann_star(left, right, gamma: float):
    """left/right = (rho, u, p); returns (p*, u*)."""
    ps, us = ctypes.c_double(), ctypes.c_double()
    rc = lib().oracle_riemann_star(*map(float, left), *map(float, right), float(gamma),
                                   ctypes.byref(ps), ctypes.byref(us))
    if rc:
        raise ValueError("vacuum generated")
    return ps.value, us.value


def riemann_sample(left, right, gamma: float, S):
    S = np.ascontiguousarray(S, dtype=np.float64)
    rho, u, p = (np.zeros_like(S) for _ in range(3))
    rc = lib().oracle_riemann_sample(*map(float, left), *map(float, right), float(gamma),
                                     _p(S), S.size, _p(rho), _p(u), _p(p))
    if rc:
        raise ValueError("vacuum generated")
    return rho, u, p


def pair_field(d: int, e: int) -> int:
    return W_F1 + 5 * PAIRS.index((d, e))


# test instrumentation: which guard branches of the method a run took
BRANCHES = ("prim_dens_floor", "prim_pres_floor", "trace_dens_floor", "trace_pres_floor", "davis",
            "revert_stage1", "revert_stage2", "corrected_pres_floor")


def branch_hits(reset: bool = True) -> dict:
    """Counts of the guard branches taken since the last reset (and reset them)."""
    out = (ctypes.c_long * len(BRANCHES))()
    lib().oracle_branch_hits(out, len(BRANCHES), int(reset))
    return dict(zip(BRANCHES, (int(v) for v in out)))


def set_wall_r11(on: bool) -> None:
    """R11 (impermeable reflecting faces) on (default) or off."""
    lib().oracle_set_wall_r11(int(bool(on)))
