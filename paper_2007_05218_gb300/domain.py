"""Decomposition of one domain into boxes (the paper's MultiFab of Fabs, §2).

`decompose` cuts a problem's interior into a grid of boxes and returns the
sub-problems with the neighbour table `hydro_set_neighbors` takes: internal
faces are linked to the adjacent box, periodic domain faces to the box at the
other end, and the remaining faces keep the domain's boundary condition.
`assemble` puts the boxes' interiors back together.
"""
from __future__ import annotations

import itertools

import numpy as np

from .inputs import Problem


def decompose(problem: Problem, cuts):
    """cuts = (xs, ys, zs): lists of box extents along each axis (summing to the
    domain's extents).  Returns (problems, neighbors[nboxes][6], origins)."""
    nx, ny, nz = problem.shape
    for a, (c, n) in enumerate(zip(cuts, (nx, ny, nz))):
        if sum(c) != n or min(c) < 4:
            raise ValueError(f"cuts along axis {a} must be >= 4 zones each and sum to {n}")
    starts = [np.concatenate([[0], np.cumsum(c)[:-1]]).astype(int) for c in cuts]
    counts = [len(c) for c in cuts]
    index = {}
    boxes, origins = [], []
    for k, j, i in itertools.product(range(counts[2]), range(counts[1]), range(counts[0])):
        index[(i, j, k)] = len(boxes)
        o = (starts[0][i], starts[1][j], starts[2][k])
        ext = (cuts[0][i], cuts[1][j], cuts[2][k])
        U = np.ascontiguousarray(problem.U[:, o[2]:o[2] + ext[2], o[1]:o[1] + ext[1], o[0]:o[0] + ext[0]])
        boxes.append(Problem(problem.name, U, problem.dx, problem.gamma, problem.cfl, problem.bc,
                             problem.nsteps, dict(problem.meta)))
        origins.append(o)
    nbr = -np.ones((len(boxes), 6), dtype=np.int32)
    for (i, j, k), b in index.items():
        pos = [i, j, k]
        for a in range(3):
            for side in (0, 1):
                q = list(pos)
                q[a] += -1 if side == 0 else 1
                if 0 <= q[a] < counts[a]:
                    nbr[b, 2 * a + side] = index[tuple(q)]
                elif problem.bc[2 * a + side] == "periodic":
                    q[a] %= counts[a]
                    nbr[b, 2 * a + side] = index[tuple(q)]
    return boxes, nbr, origins


def assemble(shape, interiors, origins) -> np.ndarray:
    """Inverse of decompose for interior states: [5][nz][ny][nx]."""
    nx, ny, nz = shape
    out = np.zeros((5, nz, ny, nx))
    for U, o in zip(interiors, origins):
        ez, ey, ex = U.shape[1:]
        out[:, o[2]:o[2] + ez, o[1]:o[1] + ey, o[0]:o[0] + ex] = U
    return out
