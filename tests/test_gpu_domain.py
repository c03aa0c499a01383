"""Boxes of one domain: ghost zones of internal faces filled from the
neighbouring box, one shared dt.  A domain split into boxes must advance
bitwise like the same domain in one box (and so match the oracle)."""
import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import domain, hydro, inputs


def run_whole(pr, nsteps, precision=hydro.HYDRO_FP64):
    B = hydro.Boxes([pr], precision=precision)
    B.step(nsteps)
    B.sync()
    U, t = B.interior(0), B.time()[0]
    B.close()
    return U, t


def run_split(pr, cuts, nsteps, precision=hydro.HYDRO_FP64):
    boxes, nbr, origins = domain.decompose(pr, cuts)
    B = hydro.Boxes(boxes, precision=precision)
    hydro.hydro_set_neighbors(B.h, nbr)
    hydro.hydro_set_shared_dt(B.h, True)
    B.step(nsteps)
    B.sync()
    U = domain.assemble(pr.shape, [B.interior(k) for k in range(B.nboxes)], origins)
    t = B.time()
    B.close()
    return U, t


def test_decompose_links_and_reassembles():
    pr = inputs.kelvin_helmholtz((24, 16, 12), seed=1)  # periodic x, z; reflect y
    boxes, nbr, origins = domain.decompose(pr, ([10, 14], [8, 8], [12]))
    assert len(boxes) == 4
    np.testing.assert_array_equal(domain.assemble(pr.shape, [b.U for b in boxes], origins), pr.U)
    # box 0 = (x0, y0): x neighbours wrap to box 1 on both sides, y-hi is box 2, y-lo a wall
    assert list(nbr[0]) == [1, 1, -1, 2, 0, 0]
    with pytest.raises(ValueError):
        domain.decompose(pr, ([10, 10], [16], [12]))


@pytest.mark.gpu
@pytest.mark.parametrize("name,make,cuts,nsteps,precision", [
    ("density_wave", lambda: inputs.density_wave((24, 20, 16), seed=3), ([10, 14], [12, 8], [16]), 10,
     hydro.HYDRO_FP64),
    ("shear_layer", lambda: inputs.kelvin_helmholtz((24, 32, 16), seed=4), ([12, 12], [16, 16], [8, 8]), 8,
     hydro.HYDRO_FP64),
    ("sedov_mixed", lambda: inputs.sedov((24, 24, 24), seed=2), ([12, 12], [12, 12], [12, 12]), 12,
     hydro.HYDRO_MIXED),
])
def test_split_domain_advances_like_one_box(name, make, cuts, nsteps, precision):
    pr = make()
    whole, t_whole = run_whole(pr, nsteps, precision)
    split, t_split = run_split(pr, cuts, nsteps, precision)
    np.testing.assert_array_equal(split, whole)
    assert np.all(t_split == t_whole)
    if precision == hydro.HYDRO_FP64:
        Uo, to, _, rc = oracle.run(pr, nsteps=nsteps, nthreads=8)
        err = max(np.max(np.abs(split[v] - Uo[v])) / np.max(np.abs(Uo[v])) for v in range(5))
        assert err <= 1e-10


@pytest.mark.gpu
def test_neighbour_tables_are_validated():
    pr = inputs.density_wave((24, 20, 16), seed=3)
    boxes, nbr, _ = domain.decompose(pr, ([12, 12], [20], [16]))
    other = inputs.density_wave((12, 10, 16), seed=3)
    B = hydro.Boxes(boxes + [other])
    bad = np.vstack([nbr, -np.ones((1, 6), np.int32)])
    bad[0, 0] = 2  # box 2 has other extents across an x face
    with pytest.raises(hydro.HydroError):
        hydro.hydro_set_neighbors(B.h, bad)
    bad[0, 0] = 7  # out of range
    with pytest.raises(hydro.HydroError):
        hydro.hydro_set_neighbors(B.h, bad)
    B.close()
