"""Batched uneven boxes in one launch per stage (work tables), CUDA-graph
replay of a step and the launch autotuner, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu
G = hydro.HYDRO_NG


def rel_linf(a, b):
    return max(np.max(np.abs(a[v] - b[v])) / np.max(np.abs(b[v])) for v in range(5))


def rel_l1(a, b):
    return np.sum(np.abs(a - b)) / np.sum(np.abs(b))


def _run(problems, nsteps, graphs=True, tune=False, precision=hydro.HYDRO_FP64):
    B = hydro.Boxes(problems, precision=precision)
    hydro.hydro_use_graphs(B.h, graphs)
    tuned = hydro.hydro_autotune(B.h, reps=2) if tune else None
    t0 = B.time()
    B.step(nsteps)
    B.sync()
    out = [B.interior(b) for b in range(B.nboxes)]
    t = B.time()
    B.close()
    return out, t, t0, tuned


def test_graph_replay_matches_direct_launches_bitwise():
    probs = inputs.sedov_batch(5, seed=2, nsteps=4, edges=(12, 16, 24))
    a, ta, _, _ = _run(probs, 4, graphs=True)
    b, tb, _, _ = _run(probs, 4, graphs=False)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(ta, tb)


@pytest.mark.parametrize("precision", [hydro.HYDRO_FP64, hydro.HYDRO_MIXED])
def test_autotune_keeps_state_and_results(precision):
    probs = inputs.sedov_batch(6, seed=4, nsteps=3, edges=(12, 16, 20, 24))
    a, ta, t0, tuned = _run(probs, 3, tune=True, precision=precision)
    b, tb, _, _ = _run(probs, 3, tune=False, precision=precision)
    assert np.all(t0 == 0.0)  # tuning did not advance time
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    names = {t[0] for t in tuned}
    # FP32 boxes run the fused line stage in place of slopes, tracing and the normal solves
    staged = ({"slopes", "trace", "riemann", "ctu1", "ctu2"} if precision == hydro.HYDRO_FP64
              else {"line_x", "line_yz", "ctu1_line", "ctu2_line"})
    assert {"prim"} | staged <= names
    assert all(t[2] in (64, 128, 256) and t[3] in (0, 1) and t[4] > 0 for t in tuned)


def test_batch_512_sedov_boxes_against_oracle_samples():
    """The batched configuration: 512 Sedov boxes, edges from {16,24,32,48,64},
    30 steps in one handle; three seeded boxes re-run by the oracle."""
    probs = inputs.sedov_batch(512, seed=0, nsteps=30)
    outs, times, _, _ = _run(probs, 30, tune=True)
    rng = np.random.default_rng(0)
    for k in rng.choice(512, 3, replace=False):
        pr = probs[k]
        Uo, to, _, rc = oracle.run(pr, nsteps=30, nthreads=16)
        assert rc == 0
        assert rel_linf(outs[k], Uo) <= 1e-10, (k, pr.shape)
        assert times[k] == pytest.approx(to, rel=1e-12)


def test_batch_512_sedov_mixed_against_fp64():
    probs = inputs.sedov_batch(512, seed=0, nsteps=30)
    a, _, _, _ = _run(probs, 30, precision=hydro.HYDRO_FP64)
    m, _, _, _ = _run(probs, 30, precision=hydro.HYDRO_MIXED)
    rho = max(rel_l1(m[k][0], a[k][0]) for k in range(512))
    E = max(rel_l1(m[k][4], a[k][4]) for k in range(512))
    print(f"512 Sedov boxes, 30 steps: worst box rel L1 mixed vs FP64: rho {rho:.3e}, E {E:.3e}")
    assert rho <= 1e-5 and E <= 1e-5
