"""Seeded synthetic initial conditions for the hydro update.

This module is the one piece of code shared by the CUDA path and the oracle:
it only *builds inputs* (initial conserved states, zone widths, boundary
conditions) and holds none of the update's arithmetic.  Random numbers come
from a counter-based generator keyed by (seed, box, counter) so that a zone's
value never depends on traversal order or on how many boxes are generated.

Workload families follow the paper's benchmark style: the Sedov-Taylor blast
wave of §4.A ("Blast Wave"), plus the shock tube, smooth density wave and
Kelvin-Helmholtz shear layer used to exercise the same hydro path.

Generator: the SplitMix64 finaliser (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to
    z = seed * 0x9E3779B97F4A7C15 + (box << 40) + counter   (mod 2**64)
and mapped to [0, 1) by its top 53 bits.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

BC_NAMES = ("periodic", "outflow", "reflect")

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def uniform01(seed: int, box: int, counter) -> np.ndarray:
    """Counter-based uniform numbers in [0, 1); `counter` is any int array (< 2**40)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) * _GOLDEN + (np.uint64(box) << np.uint64(40)) + c
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Problem:
    """One box: interior conserved state U[5][nz][ny][nx] = (rho, rho*u, rho*v, rho*w, E)."""
    name: str
    U: np.ndarray
    dx: tuple
    gamma: float
    cfl: float
    bc: tuple  # (xlo, xhi, ylo, yhi, zlo, zhi) names from BC_NAMES
    nsteps: int
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        """(nx, ny, nz)."""
        return (self.U.shape[3], self.U.shape[2], self.U.shape[1])

    @property
    def zones(self) -> int:
        return int(self.U.shape[1] * self.U.shape[2] * self.U.shape[3])


def _as_shape(n):
    if np.isscalar(n):
        return (int(n),) * 3
    return tuple(int(v) for v in n)


def _conserved(rho, u, v, w, p, gamma):
    U = np.empty((5,) + rho.shape, dtype=np.float64)
    U[0] = rho
    U[1] = rho * u
    U[2] = rho * v
    U[3] = rho * w
    U[4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return U


def _centres(n, lo, d):
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * d


def sod(n=32, axis=0, flip=False, gamma=1.4, cfl=0.5, nsteps=20) -> Problem:
    """Sod shock tube along `axis` in [0,1] (zone width 1/n_axis on every axis).

    Left state rho=1, p=1; right state rho=0.125, p=0.1; u=0.  The jump sits on
    the face at x=0.5.  `flip` swaps the two sides (the mirror image).  Outflow
    on all faces.
    """
    nx, ny, nz = _as_shape(n)
    shape = (nz, ny, nx)
    na = (nx, ny, nz)[axis]
    d = 1.0 / na
    xc = _centres(na, 0.0, d)
    left = xc < 0.5
    if flip:
        left = ~left
    bshape = [1, 1, 1]
    bshape[2 - axis] = na
    left = np.broadcast_to(left.reshape(bshape), shape)
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros(shape)
    U = _conserved(rho, z, z, z, p, gamma)
    return Problem("sod", U, (d, d, d), gamma, cfl, ("outflow",) * 6, nsteps,
                   {"axis": axis, "flip": flip})


def density_wave(n=256, seed=0, gamma=5.0 / 3.0, cfl=0.5, nsteps=50, noise=1e-3,
                 amp=0.1, vel=(1.0, 0.5, 0.25), box=0) -> Problem:
    """Smooth density wave rho = 1 + amp*sin(2*pi*(x+y+z)) on [0,1)^3, periodic.

    Velocity is uniform `vel`; p = 1 + noise*U(-1,1) per zone (seeded).  Each
    axis spans [0,1) with n_axis zones; rho is sampled at zone centres.
    """
    nx, ny, nz = _as_shape(n)
    dx, dy, dz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    x = _centres(nx, 0.0, dx)[None, None, :]
    y = _centres(ny, 0.0, dy)[None, :, None]
    zc = _centres(nz, 0.0, dz)[:, None, None]
    rho = 1.0 + amp * np.sin(2.0 * np.pi * (x + y + zc))
    shape = (nz, ny, nx)
    rho = np.broadcast_to(rho, shape)
    if noise:
        r = uniform01(seed, box, np.arange(nx * ny * nz, dtype=np.uint64)).reshape(shape)
        p = 1.0 + noise * (2.0 * r - 1.0)
    else:
        p = np.ones(shape)
    U = _conserved(rho, np.full(shape, vel[0]), np.full(shape, vel[1]),
                   np.full(shape, vel[2]), p, gamma)
    return Problem("density_wave", U, (dx, dy, dz), gamma, cfl, ("periodic",) * 6,
                   nsteps, {"seed": seed, "noise": noise, "amp": amp, "vel": tuple(vel)})


SEDOV_DEPOSIT_ZONES = 33  # integer offsets with a^2+b^2+c^2 <= 4


def sedov(n=(32, 32, 32), seed=0, box=0, gamma=1.4, cfl=0.5, nsteps=30, dx=1.0 / 64.0,
          energy=1.0, p_ambient=1e-5) -> Problem:
    """Sedov-style blast (the paper's §4.A benchmark) in one box.

    Ambient rho=1, p=p_ambient, u=0, cubic zones of width dx, outflow BCs.
    The centre is a zone centre drawn uniformly with at least 4 zones to every
    face; `energy` is spread evenly over the 33 zones whose centres lie within
    2*dx of it (inclusive).
    """
    nx, ny, nz = _as_shape(n)
    shape = (nz, ny, nx)
    r = uniform01(seed, box, np.arange(3, dtype=np.uint64) + np.uint64(1 << 39))
    centre = []
    for a, na in enumerate((nx, ny, nz)):
        lo, hi = 4, na - 5
        if hi < lo:
            raise ValueError("sedov box needs at least 9 zones per axis")
        centre.append(lo + min(int(r[a] * (hi - lo + 1)), hi - lo))
    ci, cj, ck = centre
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dep = (i - ci) ** 2 + (j - cj) ** 2 + (k - ck) ** 2 <= 4
    rho = np.ones(shape)
    z = np.zeros(shape)
    U = _conserved(rho, z, z, z, np.full(shape, p_ambient), gamma)
    U[4][dep] += energy / (SEDOV_DEPOSIT_ZONES * dx ** 3)
    return Problem("sedov", U, (dx, dx, dx), gamma, cfl, ("outflow",) * 6, nsteps,
                   {"seed": seed, "box": box, "centre": (ci, cj, ck)})


def kelvin_helmholtz(n=512, seed=0, gamma=1.4, cfl=0.5, nsteps=100, amp=0.01, box=0) -> Problem:
    """3D shear layer on [-1/2,1/2]^3: rho=2, u=+0.5 where |y|<0.25, else rho=1, u=-0.5.

    p=2.5; U(-amp, amp) added independently to u, v, w per zone (seeded).
    Periodic in x and z, reflecting in y.
    """
    nx, ny, nz = _as_shape(n)
    shape = (nz, ny, nx)
    dx, dy, dz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    y = _centres(ny, -0.5, dy)[None, :, None]
    inner = np.broadcast_to(np.abs(y) < 0.25, shape)
    rho = np.where(inner, 2.0, 1.0)
    u0 = np.where(inner, 0.5, -0.5)
    N = nx * ny * nz
    ctr = np.arange(N, dtype=np.uint64) * np.uint64(4)
    pert = [amp * (2.0 * uniform01(seed, box, ctr + np.uint64(c)).reshape(shape) - 1.0)
            for c in range(3)]
    U = _conserved(rho, u0 + pert[0], pert[1], pert[2], np.full(shape, 2.5), gamma)
    return Problem("kelvin_helmholtz", U, (dx, dy, dz), gamma, cfl,
                   ("periodic", "periodic", "reflect", "reflect", "periodic", "periodic"),
                   nsteps, {"seed": seed})


def uniform(n=8, rho=1.0, vel=(0.3, -0.2, 0.1), p=1.0, gamma=1.4, bc="periodic",
            cfl=0.5, nsteps=5) -> Problem:
    """A uniform state (any velocity): the scheme must keep it uniform."""
    nx, ny, nz = _as_shape(n)
    shape = (nz, ny, nx)
    U = _conserved(np.full(shape, rho), np.full(shape, vel[0]), np.full(shape, vel[1]),
                   np.full(shape, vel[2]), np.full(shape, p), gamma)
    return Problem("uniform", U, (1.0 / nx, 1.0 / ny, 1.0 / nz), gamma, cfl, (bc,) * 6, nsteps)


def checkerboard(n=(8, 6, 4), rho0=1.0, amp=0.1, vel=(1.0, -0.6, 0.35), p=1e-4, gamma=1.4, cfl=0.9,
                 nsteps=3) -> Problem:
    """Density rho0 + amp (-1)^(i+j+k) carried by a uniform velocity at uniform
    pressure, periodic; even extents, so that every zone is a local extremum
    of the density along every axis (also across the periodic seams)."""
    nx, ny, nz = _as_shape(n)
    if nx % 2 or ny % 2 or nz % 2:
        raise ValueError("checkerboard extents must be even")
    shape = (nz, ny, nx)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rho = rho0 + amp * (1.0 - 2.0 * ((i + j + k) % 2))
    U = _conserved(rho, np.full(shape, vel[0]), np.full(shape, vel[1]), np.full(shape, vel[2]),
                   np.full(shape, p), gamma)
    return Problem("checkerboard", U, (1.0 / nx, 1.0 / ny, 1.0 / nz), gamma, cfl, ("periodic",) * 6, nsteps,
                   {"rho0": rho0, "amp": amp, "vel": tuple(vel), "p": p})


def shear_cold(n=(16, 16, 8), seed=3, p=0.02, amp=0.5, gamma=1.4, cfl=0.5, nsteps=10) -> Problem:
    """A low-pressure shear layer (rho 2 inside |y| < 1/4, else 1; u = +-1/2)
    with large seeded velocity noise U(-amp, amp) on u, v, w: the transverse
    corrections of some face states come out with p <= 0 on the first step.
    Periodic x, z; reflecting y."""
    nx, ny, nz = _as_shape(n)
    shape = (nz, ny, nx)
    y = _centres(ny, -0.5, 1.0 / ny)
    inside = (np.abs(y) < 0.25)[None, :, None] & np.ones(shape, dtype=bool)
    N = nx * ny * nz
    ctr = np.arange(N, dtype=np.uint64) * np.uint64(3)
    pert = [amp * (2.0 * uniform01(seed, 0, ctr + np.uint64(c)).reshape(shape) - 1.0) for c in range(3)]
    rho = np.where(inside, 2.0, 1.0)
    u = np.where(inside, 0.5, -0.5) + pert[0]
    U = _conserved(rho, u, pert[1], pert[2], np.full(shape, p), gamma)
    return Problem("shear_cold", U, (1.0 / nx, 1.0 / ny, 1.0 / nz), gamma, cfl,
                   ("periodic", "periodic", "reflect", "reflect", "periodic", "periodic"), nsteps, {"seed": seed})


def vacuum_ball(n=(16, 16, 16), radius=0.3, rho_vac=1e-14, p_vac=1e-14, gamma=1.4, cfl=0.5,
                nsteps=10) -> Problem:
    """A ball of gas at rest (rho = 1, p = 1, radius `radius` on [-1/2,1/2]^3)
    in a near vacuum whose density and pressure lie below the method's floors;
    outflow boundaries."""
    nx, ny, nz = _as_shape(n)
    shape = (nz, ny, nx)
    x, y, z = _centres(nx, -0.5, 1.0 / nx), _centres(ny, -0.5, 1.0 / ny), _centres(nz, -0.5, 1.0 / nz)
    r2 = z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2
    inside = r2 < radius * radius
    zero = np.zeros(shape)
    U = _conserved(np.where(inside, 1.0, rho_vac), zero, zero, zero, np.where(inside, 1.0, p_vac), gamma)
    return Problem("vacuum_ball", U, (1.0 / nx, 1.0 / ny, 1.0 / nz), gamma, cfl, ("outflow",) * 6, nsteps)


BATCH_EDGES = (16, 24, 32, 48, 64)


def sedov_batch(nboxes=512, seed=0, gamma=1.4, cfl=0.5, nsteps=30, edges=BATCH_EDGES):
    """Independent Sedov boxes whose edges are drawn iid from `edges` per axis."""
    r = uniform01(seed, 1 << 23, np.arange(3 * nboxes, dtype=np.uint64))
    out = []
    for b in range(nboxes):
        shp = tuple(edges[min(int(r[3 * b + a] * len(edges)), len(edges) - 1)] for a in range(3))
        out.append(sedov(shp, seed=seed, box=b, gamma=gamma, cfl=cfl, nsteps=nsteps))
    return out


@dataclass
class ServedRequest:
    arrival_s: float
    problem: Problem
    nsteps: int
    mixed: bool


def served_stream(nrequests=2000, seed=0, rate_per_s=200.0, edge_lo=32, edge_hi=128, steps_lo=10,
                  steps_hi=200) -> list:
    """A seeded stream of independent hydro requests: Poisson arrivals at
    `rate_per_s`, box edges uniform in [edge_lo, edge_hi] per axis, step counts
    uniform in [steps_lo, steps_hi], the initial condition drawn uniformly from
    Sod (random axis and side), Sedov (random centre) and Kelvin-Helmholtz
    (random perturbation seed), FP64 or mixed precision with equal odds."""
    r = uniform01(seed, (1 << 23) + 1, np.arange(8 * nrequests, dtype=np.uint64)).reshape(nrequests, 8)
    t = 0.0
    out = []
    span_e = edge_hi - edge_lo + 1
    span_s = steps_hi - steps_lo + 1
    for k in range(nrequests):
        t += -np.log(1.0 - r[k, 0]) / rate_per_s
        shape = tuple(edge_lo + min(int(r[k, 1 + a] * span_e), span_e - 1) for a in range(3))
        nsteps = steps_lo + min(int(r[k, 4] * span_s), span_s - 1)
        kind = min(int(r[k, 5] * 3), 2)
        sub = r[k, 6]
        if kind == 0:
            axis = min(int(sub * 3), 2)
            pr = sod(shape, axis=axis, flip=bool(int(sub * 6) % 2), nsteps=nsteps)
        elif kind == 1:
            pr = sedov(shape, seed=seed, box=k, nsteps=nsteps)
        else:
            pr = kelvin_helmholtz(shape, seed=seed + 1 + k, nsteps=nsteps)
        out.append(ServedRequest(t, pr, nsteps, bool(r[k, 7] < 0.5)))
    return out
