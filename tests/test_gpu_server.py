"""Served form on the GPU: requests of different sizes, initial conditions,
precisions and step counts share the device through continuous batching;
each result must be the same alone and in the mix (bitwise: a request's
arithmetic does not depend on its neighbours in the batch)."""
import numpy as np
import pytest

from paper_2007_05218_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu


def alone(problem, nsteps, precision):
    B = hydro.Boxes([problem], precision=precision)
    B.step(nsteps)
    B.sync()
    U = B.interior(0)
    t = B.time()[0]
    B.close()
    return U, t


def mix():
    reqs = [
        (inputs.sod((40, 8, 6), axis=0), 25, hydro.HYDRO_FP64),
        (inputs.sedov((20, 24, 18), seed=1), 30, hydro.HYDRO_MIXED),
        (inputs.kelvin_helmholtz((24, 32, 16), seed=2), 12, hydro.HYDRO_FP64),
        (inputs.density_wave((16, 20, 24), seed=3), 40, hydro.HYDRO_MIXED),
        (inputs.sod((6, 36, 8), axis=1, flip=True), 18, hydro.HYDRO_MIXED),
        (inputs.sedov((32, 16, 16), seed=4), 7, hydro.HYDRO_FP64),
        (inputs.density_wave((12, 12, 12), seed=5), 0, hydro.HYDRO_FP64),
        (inputs.kelvin_helmholtz((16, 16, 16), seed=6), 33, hydro.HYDRO_MIXED),
    ]
    return reqs


def test_each_request_is_the_same_alone_and_in_the_mix():
    reqs = mix()
    # a budget that holds only a few requests at once, so most of them queue
    srv = hydro.Server(600 * 1024 * 1024, max_active=3)
    tickets = [srv.submit(p, nsteps=n, precision=prec) for p, n, prec in reqs]
    results = [srv.wait(t, p.shape) for t, (p, n, prec) in zip(tickets, reqs)]
    st = srv.stats()
    srv.close()
    assert st["finished"] == len(reqs) and st["peak_bytes"] <= st["budget_bytes"]
    for (p, n, prec), (U, info) in zip(reqs, results):
        assert info.status == hydro.HYDRO_OK and info.steps == n
        ref, t_ref = alone(p, n, prec)
        np.testing.assert_array_equal(U, ref)
        assert info.time == t_ref


def test_a_failing_request_does_not_disturb_the_others():
    good = inputs.density_wave((16, 12, 10), seed=8)
    bad = inputs.uniform(8)
    bad.U[0, 3, 3, 3] = -1.0
    srv = hydro.Server(512 * 1024 * 1024, max_active=4)
    tg = srv.submit(good, nsteps=6)
    tb = srv.submit(bad, nsteps=3)
    U, info = srv.wait(tg, good.shape)
    Ub, info_b = srv.wait(tb, bad.shape)
    srv.close()
    assert info_b.status == hydro.HYDRO_ERR_NONPHYSICAL and Ub is None
    ref, _ = alone(good, 6, hydro.HYDRO_FP64)
    np.testing.assert_array_equal(U, ref)


def test_many_small_requests_through_few_slots():
    probs = [inputs.sedov((12, 12, 12), seed=k, box=k) for k in range(24)]
    srv = hydro.Server(1 << 30, max_active=5)
    tickets = [srv.submit(p, nsteps=4 + k % 5) for k, p in enumerate(probs)]
    res = [srv.wait(t, p.shape) for t, p in zip(tickets, probs)]
    st = srv.stats()
    srv.close()
    assert st["finished"] == 24 and st["active"] == 0 and st["bytes_in_use"] == 0
    for k, (p, (U, info)) in enumerate(zip(probs, res)):
        ref, _ = alone(p, 4 + k % 5, hydro.HYDRO_FP64)
        np.testing.assert_array_equal(U, ref)
