"""FP64 CUDA path vs the oracle, through the C ABI (needs a GB300).

Tolerance: relative L-infinity per conserved field, max|gpu - oracle| / max|oracle|,
at most 1e-10 after 10 steps (field-max normalisation, since pointwise relative
error is undefined where a momentum component crosses zero).  Intermediates of
one step are compared field by field on the regions the step defines.
"""
import numpy as np
import pytest

import oracle
from paper_2007_05218_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10
G = hydro.HYDRO_NG


def torch_mod():
    import torch
    return torch


def rel_linf(a, b):
    out = []
    for v in range(a.shape[0]):
        scale = np.max(np.abs(b[v]))
        diff = np.max(np.abs(a[v] - b[v]))
        out.append(diff / scale if scale > 0 else diff)
    return np.array(out)


def run_gpu(problems, nsteps):
    B = hydro.Boxes(problems)
    B.step(nsteps)
    B.sync()
    out = [B.interior(b) for b in range(B.nboxes)]
    t = B.time()
    B.close()
    return out, t


CASES = {
    "sod_x": lambda: inputs.sod((32, 6, 5), axis=0),
    "sod_y": lambda: inputs.sod((5, 24, 6), axis=1),
    "sod_z_mirror": lambda: inputs.sod((6, 5, 20), axis=2, flip=True),
    "density_wave_ragged": lambda: inputs.density_wave((20, 12, 9), seed=3),
    "sedov": lambda: inputs.sedov((17, 16, 18), seed=2),
    "kelvin_helmholtz_reflect_y": lambda: inputs.kelvin_helmholtz((12, 16, 10), seed=4),
    "uniform_outflow": lambda: inputs.uniform((8, 9, 10), bc="outflow"),
    "uniform_reflect": lambda: inputs.uniform((7, 6, 5), vel=(0.0, 0.0, 0.0), bc="reflect"),
    "minimum_box_4cubed": lambda: inputs.density_wave((4, 4, 4), seed=5),
    "long_thin_x": lambda: inputs.kelvin_helmholtz((300, 4, 6), seed=6),
    "long_thin_z": lambda: inputs.density_wave((4, 6, 200), seed=7),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_matches_oracle_after_10_steps(name):
    pr = CASES[name]()
    Uo, to, dts, rc = oracle.run(pr, nsteps=10)
    assert rc == 0
    (Ug,), tg = run_gpu([pr], 10)
    err = rel_linf(Ug, Uo)
    assert np.all(err <= TOL), err
    assert tg[0] == pytest.approx(to, rel=1e-12)


@pytest.mark.parametrize("name", ["density_wave_ragged", "sedov", "kelvin_helmholtz_reflect_y"])
def test_dt_matches_oracle(name):
    pr = CASES[name]()
    box = oracle.box_of(pr)
    dt_o = oracle.compute_dt(box, oracle.embed(pr.U))
    B = hydro.Boxes([pr])
    dt_g = B.compute_dt().cpu().numpy()[0]
    B.close()
    assert dt_g == pytest.approx(dt_o, rel=1e-14)


def _regions(n):
    """Slices (k, j, i order) of every intermediate field's defined region."""
    def sl(kind, a):
        return {"all": slice(0, n[a] + 2 * G), "ext": slice(G - 1, G + n[a] + 1),
                "face": slice(G, G + n[a] + 1), "int": slice(G, G + n[a])}[kind]

    def reg(kinds):
        return (sl(kinds[2], 2), sl(kinds[1], 1), sl(kinds[0], 0))

    out = {}
    for f in range(5):
        out[f] = ("q", reg(("all",) * 3))
    out[oracle.W_C] = ("c", reg(("all",) * 3))
    out[oracle.W_CHI] = ("chi", reg(("ext",) * 3))
    for d in range(3):
        for m in range(5):
            out[oracle.W_QM + 5 * d + m] = (f"qm{d}{m}", reg(("ext",) * 3))
            out[oracle.W_QP + 5 * d + m] = (f"qp{d}{m}", reg(("ext",) * 3))
            k = ["ext"] * 3
            k[d] = "face"
            out[oracle.W_F0 + 5 * d + m] = (f"f0{d}{m}", reg(k))
            k = ["int"] * 3
            k[d] = "face"
            out[oracle.W_F + 5 * d + m] = (f"f{d}{m}", reg(k))
    for p, (d, e) in enumerate(oracle.PAIRS):
        f = 3 - d - e
        k = [None] * 3
        k[d], k[e], k[f] = "face", "int", "ext"
        for m in range(5):
            out[oracle.W_F1 + 5 * p + m] = (f"f1{d}{e}{m}", reg(k))
    return out


@pytest.mark.parametrize("name", ["sedov", "kelvin_helmholtz_reflect_y", "sod_y"])
def test_every_stage_matches_oracle_on_one_step(name):
    torch = torch_mod()
    pr = CASES[name]()
    box = oracle.box_of(pr)
    Ug = oracle.embed(pr.U)
    oracle.fill_ghosts(box, Ug)
    dt = oracle.compute_dt(box, Ug)
    rc, W = oracle.step(box, Ug, dt, dump=True)
    assert rc == 0
    B = hydro.Boxes([pr])
    B.step(1, dt=torch.tensor([dt], dtype=torch.float64, device="cuda"))
    B.sync()
    Wg = B.field_view(0, 0, oracle.W_NFIELDS).cpu().numpy()
    nf = hydro.hydro_debug_fields(B.descs, 0)[1]
    recips = B.field_view(0, nf - 2, 2).cpu().numpy()  # 1/c and c/rho of each zone (FP64 boxes)
    Ugpu = B.interior(0)
    B.close()
    bad = []
    regions = _regions(pr.shape)
    reg = regions[oracle.W_C][1]
    c, rho = W[oracle.W_C][reg], W[0][reg]
    assert np.max(np.abs(recips[0][reg] * c - 1.0)) <= 1e-13
    assert np.max(np.abs(recips[1][reg] * rho / c - 1.0)) <= 1e-13
    for f, (label, reg) in regions.items():
        a, b = Wg[f][reg], W[f][reg]
        # scale: the largest magnitude among the five fields of the same group
        # (one state or flux), so that components the oracle holds at exactly
        # zero (transverse momentum fluxes of a shock tube) are judged against
        # their group's size; fused multiply-adds leave ~1e-17 residues there
        g0 = f if f < 5 else oracle.W_QM + (f - oracle.W_QM) // 5 * 5
        group = range(0, 5) if f < 5 else ([f] if f in (oracle.W_C, oracle.W_CHI) else range(g0, g0 + 5))
        scale = max(np.max(np.abs(W[h][regions[h][1]])) for h in group)
        diff = np.max(np.abs(a - b))
        if diff > 1e-11 * scale:
            bad.append((label, diff, scale))
    assert not bad, bad[:10]
    assert np.all(rel_linf(Ugpu, oracle.interior(Ug)) <= 1e-12)


def test_batch_of_uneven_boxes_matches_each_box_alone():
    probs = inputs.sedov_batch(6, seed=5, nsteps=5, edges=(12, 16, 20))
    outs, times = run_gpu(probs, 5)
    for k, pr in enumerate(probs):
        Uo, to, _, rc = oracle.run(pr, nsteps=5)
        assert rc == 0
        assert np.all(rel_linf(outs[k], Uo) <= TOL)
        assert times[k] == pytest.approx(to, rel=1e-12)
        (alone,), _ = run_gpu([pr], 5)
        np.testing.assert_array_equal(alone, outs[k])  # same kernels: bitwise equal


def test_upload_download_roundtrip_is_exact():
    probs = [inputs.density_wave((12, 8, 6), seed=1), inputs.sod((10, 5, 4))]
    descs = [hydro.desc_of(p) for p in probs]
    B = hydro.Boxes(descs)
    host = np.concatenate([p.U.ravel() for p in probs])
    hydro.hydro_upload(B.h, host)
    for k, p in enumerate(probs):
        np.testing.assert_array_equal(B.interior(k), p.U)
    back = np.zeros_like(host)
    hydro.hydro_download(B.h, back)
    np.testing.assert_array_equal(back, host)
    with pytest.raises(hydro.HydroError):
        hydro.hydro_upload(B.h, host[:-1])
    B.close()


def test_ghost_fill_matches_oracle_exactly():
    for pr in (CASES["kelvin_helmholtz_reflect_y"](), CASES["sod_x"](), CASES["density_wave_ragged"]()):
        box = oracle.box_of(pr)
        Ug = oracle.embed(pr.U)
        oracle.fill_ghosts(box, Ug)
        B = hydro.Boxes([pr])
        B.fill_ghosts()
        torch_mod().cuda.synchronize()
        np.testing.assert_array_equal(B.ghosted(0), Ug)
        B.close()


def test_nonphysical_state_is_reported_on_sync():
    pr = inputs.uniform(8)
    pr.U[0, 3, 3, 3] = -1.0
    B = hydro.Boxes([pr])
    B.step(1)
    with pytest.raises(hydro.HydroError) as e:
        B.sync()
    assert e.value.code == hydro.HYDRO_ERR_NONPHYSICAL
    assert B.sync() == hydro.HYDRO_OK  # flags are cleared once reported
    B.close()


def test_zero_steps_is_a_no_op():
    pr = CASES["sedov"]()
    B = hydro.Boxes([pr])
    B.step(0)
    B.sync()
    np.testing.assert_array_equal(B.interior(0), pr.U)
    B.close()


def _window(U, bc, lo, w, ghosts):
    """Interior window [lo, lo+w) per axis (x,y,z) of the full interior state U
    plus `ghosts` zones per side taken with the boundary conditions' mapping."""
    nz, ny, nx = U.shape[1:]
    idx, flip = [], []
    for a, n in enumerate((nx, ny, nz)):
        r = np.arange(lo[a] - ghosts, lo[a] + w + ghosts)
        kind = bc[2 * a]
        f = np.zeros(r.size, bool)
        if kind == "periodic":
            r = r % n
        elif kind == "outflow":
            r = np.clip(r, 0, n - 1)
        else:
            f = (r < 0) | (r >= n)
            r = np.where(r < 0, -1 - r, np.where(r >= n, 2 * n - 1 - r, r))
        idx.append(r)
        flip.append(f)
    out = U[:, idx[2][:, None, None], idx[1][None, :, None], idx[0][None, None, :]].copy()
    for a in range(3):
        shape = [1, 1, 1]
        shape[2 - a] = -1
        out[1 + a] *= np.where(flip[a], -1.0, 1.0).reshape(shape)
    return out


def _full_size_windows(pr, nsteps, windows, w=12):
    """Windows lie inside the box (their ghost zones may wrap or reflect)."""
    torch = torch_mod()
    for lo in windows:
        assert all(0 <= lo[a] and lo[a] + w <= pr.shape[a] for a in range(3)), lo
    box = oracle.box_of(pr)
    dt = oracle.compute_dt(box, oracle.embed(pr.U))  # dt of the initial state, from the oracle
    B = hydro.Boxes([pr])
    B.step(nsteps, dt=torch.tensor([dt], dtype=torch.float64, device="cuda"))
    B.sync()
    lay = B.layouts[0]
    errs = []
    m = 4 * (nsteps - 1)  # extra margin: each step consumes 4 zones of halo
    for lo in windows:
        big = _window(pr.U, pr.bc, [l - m for l in lo], w + 2 * m, G)
        wb = oracle.make_box((w + 2 * m,) * 3, pr.dx, pr.gamma, pr.cfl, ("periodic",) * 6)
        for _ in range(nsteps):
            rc, _ = oracle.step(wb, big, dt, nthreads=8)
            assert rc == 0
        ref = big[:, G + m:G + m + w, G + m:G + m + w, G + m:G + m + w]
        gv = B.state_view(0)
        sl = tuple(slice(G + lo[a], G + lo[a] + w) for a in (2, 1, 0))
        got = gv[(slice(None),) + sl].cpu().numpy()
        errs.append(rel_linf(got, ref))
    sums = B.state_view(0)[:, G:-G, G:-G, G:-G].sum(dim=(1, 2, 3)).cpu().numpy()
    B.close()
    return np.array(errs), sums


def test_full_size_density_wave_256_sampled_windows():
    """The 256^3 density-wave workload, in the launch configuration the benchmark
    times: sampled windows (one wrapping the periodic corner) vs the oracle."""
    pr = inputs.density_wave(256, seed=0)
    windows = [(0, 0, 0), (244, 3, 128), (100, 244, 244), (37, 191, 64)]
    errs, sums = _full_size_windows(pr, 3, windows)
    assert np.all(errs <= TOL), errs
    U0 = pr.U.reshape(5, -1)
    drift = np.abs(sums - U0.sum(axis=1)) / np.abs(U0).sum(axis=1)
    assert np.all(drift <= 1e-13 * np.sqrt(3)), drift


def test_full_size_density_wave_conserves_over_benchmark_steps():
    pr = inputs.density_wave(256, seed=0)
    B = hydro.Boxes([pr])
    B.step(50)
    B.sync()
    sums = B.state_view(0)[:, G:-G, G:-G, G:-G].sum(dim=(1, 2, 3)).cpu().numpy()
    B.close()
    U0 = pr.U.reshape(5, -1)
    drift = np.abs(sums - U0.sum(axis=1)) / np.abs(U0).sum(axis=1)
    assert np.all(drift <= 1e-13 * np.sqrt(50)), drift


def test_largest_box_kelvin_helmholtz_512_sampled_windows():
    """The largest configured box (512^3 shear layer, reflecting y walls)."""
    pr = inputs.kelvin_helmholtz(512, seed=0)
    windows = [(0, 0, 0), (502, 502, 7), (256, 130, 300)]
    errs, _ = _full_size_windows(pr, 1, windows, w=10)
    assert np.all(errs <= TOL), errs
