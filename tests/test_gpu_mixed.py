"""Mixed precision (FP32 reconstruction/tracing/CTU/Riemann, FP64 state,
update and dt) vs the FP64 oracle, through the C ABI (needs a GB300).

Bar: relative L1 error sum|mixed - oracle| / sum|oracle| <= 1e-5 for density
and total energy, per result; conservation still to FP64 round-off (each
face flux is one value applied to both neighbours in FP64).
"""
import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu
TOL_L1 = 1e-5
G = hydro.HYDRO_NG


def rel_l1(a, b):
    return np.sum(np.abs(a - b)) / np.sum(np.abs(b))


def run(problems, nsteps, precision):
    B = hydro.Boxes(problems, precision=precision)
    B.step(nsteps)
    B.sync()
    out = [B.interior(b) for b in range(B.nboxes)]
    t = B.time()
    B.close()
    return out, t


CASES = {
    "sod_x": (lambda: inputs.sod((64, 6, 5), axis=0), 20),
    "density_wave": (lambda: inputs.density_wave((24, 20, 16), seed=3), 30),
    "sedov": (lambda: inputs.sedov((24, 24, 24), seed=2), 30),
    "kelvin_helmholtz": (lambda: inputs.kelvin_helmholtz((24, 32, 16), seed=4), 30),
    "minimum_box_4cubed": (lambda: inputs.density_wave((4, 4, 4), seed=5), 20),
    "long_thin_x": (lambda: inputs.kelvin_helmholtz((300, 4, 6), seed=6), 20),
    "long_thin_y": (lambda: inputs.density_wave((5, 130, 4), seed=7), 20),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_matches_fp64_oracle_in_l1(name):
    make, nsteps = CASES[name]
    pr = make()
    Uo, to, _, rc = oracle.run(pr, nsteps=nsteps, nthreads=8)
    assert rc == 0
    (Um,), tm = run([pr], nsteps, hydro.HYDRO_MIXED)
    err_rho, err_E = rel_l1(Um[0], Uo[0]), rel_l1(Um[4], Uo[4])
    print(f"{name}: {nsteps} steps, rel L1 rho {err_rho:.3e}, E {err_E:.3e}")
    assert err_rho <= TOL_L1 and err_E <= TOL_L1, (err_rho, err_E)
    # dt is reduced in FP64 from the FP64 state, so the clocks stay close too
    assert tm[0] == pytest.approx(to, rel=1e-4)


@pytest.mark.parametrize("make", [lambda: inputs.density_wave((20, 12, 16), seed=7),
                                  lambda: inputs.kelvin_helmholtz(16, seed=2)])
def test_mixed_conserves_to_fp64_roundoff(make):
    pr = make()
    pr.bc = ("periodic",) * 6
    nsteps = 20
    (Um,), _ = run([pr], nsteps, hydro.HYDRO_MIXED)
    U0 = pr.U
    for v in range(5):
        drift = abs(Um[v].sum() - U0[v].sum()) / np.abs(U0[v]).sum()
        assert drift <= 1e-13 * np.sqrt(nsteps), (v, drift)


def test_mixed_and_fp64_boxes_share_one_handle():
    probs = inputs.sedov_batch(4, seed=9, nsteps=6, edges=(12, 16, 20))
    descs = [hydro.desc_of(p, hydro.HYDRO_MIXED if k % 2 else hydro.HYDRO_FP64) for k, p in enumerate(probs)]
    B = hydro.Boxes(descs)
    for k, p in enumerate(probs):
        B.set_interior(k, p.U)
    B.step(6)
    B.sync()
    both = [B.interior(k) for k in range(len(probs))]
    B.close()
    for k, p in enumerate(probs):
        prec = hydro.HYDRO_MIXED if k % 2 else hydro.HYDRO_FP64
        (alone,), _ = run([p], 6, prec)
        np.testing.assert_array_equal(both[k], alone)


def test_mixed_stage_fields_are_fp32():
    pr = CASES["kelvin_helmholtz"][0]()
    B = hydro.Boxes([pr], precision=hydro.HYDRO_MIXED)
    B.step(1)
    B.sync()
    q = B.field_view(0, 0, 5)
    assert str(q.dtype) == "torch.float32"
    rho = q[0, G:-G, G:-G, G:-G].double().cpu().numpy()
    # primitive density of the state the step started from, rounded to FP32
    np.testing.assert_allclose(rho, pr.U[0], rtol=1e-7)
    B.close()


def test_mixed_full_size_shear_layer_512_against_fp64_path():
    """The 512^3 shear layer of the mixed-vs-FP64 configuration, 100 steps:
    the mixed result against the FP64 GPU path (itself checked against the
    oracle on sampled windows of the same box)."""
    import torch
    pr = inputs.kelvin_helmholtz(512, seed=0)
    nsteps = 100
    B = hydro.Boxes([pr], precision=hydro.HYDRO_FP64)
    B.step(nsteps)
    B.sync()
    ref = B.state_view(0)[:, G:-G, G:-G, G:-G][[0, 4]].cpu().numpy()
    t_ref = B.time()[0]
    B.close()
    del B
    torch.cuda.empty_cache()
    M = hydro.Boxes([pr], precision=hydro.HYDRO_MIXED)
    M.step(nsteps)
    M.sync()
    got = M.state_view(0)[:, G:-G, G:-G, G:-G][[0, 4]].cpu().numpy()
    t_m = M.time()[0]
    sums = M.state_view(0)[:, G:-G, G:-G, G:-G].sum(dim=(1, 2, 3)).cpu().numpy()
    M.close()
    err_rho, err_E = rel_l1(got[0], ref[0]), rel_l1(got[1], ref[1])
    print(f"KH 512^3, {nsteps} steps: mixed vs FP64 rel L1 rho {err_rho:.3e}, E {err_E:.3e}")
    assert err_rho <= TOL_L1 and err_E <= TOL_L1, (err_rho, err_E)
    assert t_m == pytest.approx(t_ref, rel=1e-4)
    U0 = pr.U.reshape(5, -1)
    for v in (0, 4):  # reflecting y walls conserve mass and energy
        assert abs(sums[v] - U0[v].sum()) <= 1e-13 * np.sqrt(nsteps) * np.abs(U0[v]).sum() * 3


def _one_step_fields(pr, fuse, riemann=0):
    import torch
    box = oracle.box_of(pr)
    Ug = oracle.embed(pr.U)
    oracle.fill_ghosts(box, Ug)
    dt = oracle.compute_dt(box, Ug)
    B = hydro.Boxes([pr], precision=hydro.HYDRO_MIXED, riemann=riemann)
    hydro.hydro_fuse_lines(B.h, fuse)
    B.step(1, dt=torch.tensor([dt], dtype=torch.float64, device="cuda"))
    B.sync()
    # zones a field does not cover hold whatever the scratch held, signalling
    # NaN patterns included, whose widening raises numpy's invalid flag; only
    # the covered regions are compared
    with np.errstate(invalid="ignore"):
        W = B.field_view(0, 0, oracle.W_NFIELDS).cpu().numpy().astype(np.float64)
    U = B.interior(0)
    B.close()
    return W, U


@pytest.mark.parametrize("riemann", [hydro.HYDRO_RIEMANN_HLLC, hydro.HYDRO_RIEMANN_TWO_SHOCK])
@pytest.mark.parametrize("make", [lambda: inputs.sedov((31, 29, 17), seed=6),
                                  lambda: inputs.density_wave((4, 5, 6), seed=2),
                                  lambda: inputs.kelvin_helmholtz((60, 4, 33), seed=3)])
def test_fused_line_stage_matches_the_separate_stages(make, riemann):
    """The fused line kernel (slopes + parabolas + tracing + normal Riemann
    solves per axis, FP32) computes what the separate FP32 stages compute:
    the edge states, normal fluxes and updated state of one step agree to
    FP32 rounding (the two builds may fuse multiply-adds differently) on
    rows that do not fill whole warps and columns that do not fill whole
    segments."""
    pr = make()
    Wf, Uf = _one_step_fields(pr, True, riemann)
    Ws, Us = _one_step_fields(pr, False, riemann)
    G = hydro.HYDRO_NG
    ext = tuple(slice(G - 1, G + n + 1) for n in pr.shape[::-1])
    for base in (oracle.W_QM, oracle.W_QP, oracle.W_F0):
        for g in range(3):
            blk = slice(base + 5 * g, base + 5 * g + 5)
            a, b = Wf[blk][(slice(None),) + ext], Ws[blk][(slice(None),) + ext]
            if base == oracle.W_F0:   # fluxes are defined on faces 0..n along their axis
                sl = [slice(None)] * 4
                sl[3 - g] = slice(1, pr.shape[g] + 2)
                a, b = a[tuple(sl)], b[tuple(sl)]
            scale = np.max(np.abs(b)) + 1e-30
            assert np.all(np.isfinite(a)), (base, g)
            assert np.max(np.abs(a - b)) <= 1e-6 * scale, (base, g)
    mom = max(np.max(np.abs(Us[v])) for v in (1, 2, 3))   # momenta judged on their common scale
    for v in range(5):
        scale = mom if v in (1, 2, 3) else np.max(np.abs(Us[v]))
        assert np.max(np.abs(Uf[v] - Us[v])) <= 1e-6 * (scale + 1e-30), v
