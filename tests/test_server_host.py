"""Host logic of the served form (admission under a memory budget, slots,
queueing, tickets, cancellation), run through the server's dry-run mode: no
GPU work, a tick completes one step of every resident request instantly and
a result equals its initial state."""
import time

import numpy as np
import pytest

from paper_2007_05218_gb300 import hydro, inputs


def footprint(problem, precision=hydro.HYDRO_FP64):
    """Bytes a resident request takes from the pool (state + scratch fields)."""
    d = hydro.desc_of(problem, precision)
    sb, wb = hydro.hydro_workspace_size([d])
    off, nf, eb = hydro.hydro_debug_fields([d], 0)
    lay = hydro.hydro_box_layout([d], 0)
    up = lambda v: (v + 255) // 256 * 256
    return up(sb) + up(nf * lay.var_stride * eb)


def wait_all(srv, tickets, shapes, timeout=20.0):
    out = {}
    for t, shp in zip(tickets, shapes):
        out[t] = srv.wait(t, shp, timeout=timeout)
    return out


def test_dry_server_runs_every_request_and_respects_the_budget():
    probs = [inputs.sod((8 + 2 * k, 6, 5)) for k in range(8)]
    big = max(footprint(p) for p in probs)
    budget = 3 * big + 64 * 1024  # room for about three resident requests (plus the tables)
    srv = hydro.Server(budget, max_active=4, dry_run=True)
    tickets = [srv.submit(p, nsteps=50 + k) for k, p in enumerate(probs)]
    res = wait_all(srv, tickets, [p.shape for p in probs])
    st = srv.stats()
    srv.close()
    assert st["finished"] == 8 and st["admitted"] == 8 and st["queued"] == 0 and st["active"] == 0
    assert st["peak_bytes"] <= st["budget_bytes"]
    assert st["bytes_in_use"] == 0
    for k, (t, p) in enumerate(zip(tickets, probs)):
        U, info = res[t]
        np.testing.assert_array_equal(U, p.U)
        assert info.status == hydro.HYDRO_OK and info.steps == 50 + k
        assert info.latency_s >= info.queued_s >= 0.0


def test_dry_server_slot_limit_and_bypass_of_a_head_that_does_not_fit():
    small = inputs.sod((8, 6, 5))
    large = inputs.sod((40, 24, 20))
    budget = footprint(large) + footprint(small) // 2 + 64 * 1024  # large fits only alone
    srv = hydro.Server(budget, max_active=8, dry_run=True)
    t_small0 = srv.submit(small, nsteps=200000)  # resident for a long while
    time.sleep(0.01)
    t_large = srv.submit(large, nsteps=1)         # must wait for the pool
    t_small1 = srv.submit(small, nsteps=1)        # fits beside small0: passes the large head
    r1 = srv.wait(t_small1, small.shape)[1]
    rl = srv.wait(t_large, large.shape)[1]
    r0 = srv.wait(t_small0, small.shape)[1]
    st = srv.stats()
    srv.close()
    assert r1.latency_s < rl.latency_s  # the small request did not queue behind the large one
    assert rl.queued_s > 0.0
    assert r0.steps == 200000 and r1.steps == 1 and rl.steps == 1
    assert st["peak_bytes"] <= st["budget_bytes"]


def test_dry_server_never_exceeds_max_active():
    probs = [inputs.sod((8, 6, 5)) for _ in range(12)]
    srv = hydro.Server(1 << 30, max_active=3, dry_run=True)
    tickets = [srv.submit(p, nsteps=2000) for p in probs]
    peak_active = 0
    while srv.stats()["finished"] < 12:
        peak_active = max(peak_active, srv.stats()["active"])
    wait_all(srv, tickets, [p.shape for p in probs])
    srv.close()
    assert 1 <= peak_active <= 3


def test_request_larger_than_the_budget_is_refused():
    large = inputs.sod((64, 32, 32))
    srv = hydro.Server(footprint(large) // 2, max_active=2, dry_run=True)
    with pytest.raises(hydro.HydroError) as e:
        srv.submit(large, nsteps=1)
    assert e.value.code == hydro.HYDRO_ERR_NOMEM
    srv.close()


def test_invalid_requests_and_tickets():
    srv = hydro.Server(1 << 28, max_active=2, dry_run=True)
    bad = inputs.sod((8, 6, 5))
    d = hydro.desc_of(bad)
    d.gamma = 0.5
    with pytest.raises(hydro.HydroError) as e:
        hydro.hydro_submit(srv.s, d, bad.U, 1)
    assert e.value.code == hydro.HYDRO_ERR_INVALID
    with pytest.raises(hydro.HydroError):
        hydro.hydro_submit(srv.s, hydro.desc_of(bad), bad.U, -1)
    t = srv.submit(bad, nsteps=0)
    U, info = srv.wait(t, bad.shape)
    np.testing.assert_array_equal(U, bad.U)
    with pytest.raises(hydro.HydroError):  # collected already
        hydro.hydro_poll(srv.s, t)
    with pytest.raises(hydro.HydroError):
        hydro.hydro_poll(srv.s, 12345)
    srv.close()


def test_server_rejects_bad_configs():
    with pytest.raises(hydro.HydroError):
        hydro.hydro_server_create(None, 1 << 20, 0, dry_run=True)
    with pytest.raises(hydro.HydroError):
        hydro.hydro_server_create(None, 1 << 20, 4, dry_run=False)  # a GPU server needs a pool
    with pytest.raises(hydro.HydroError) as e:
        hydro.hydro_server_create(None, 1024, 4096, dry_run=True)  # the tables alone do not fit
    assert e.value.code == hydro.HYDRO_ERR_NOMEM


def test_destroy_cancels_queued_requests():
    probs = [inputs.sod((8, 6, 5)) for _ in range(4)]
    srv = hydro.Server(1 << 28, max_active=1, dry_run=True)
    for p in probs:
        srv.submit(p, nsteps=10 ** 7)
    srv.close()  # returns: queued ones are cancelled, the resident one finishes
