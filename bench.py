#!/usr/bin/env python3
"""Benchmark: FP64 unsplit PPM/CTU/HLLC hydro update on one GB300.

Workload (the metric's FP64 configuration): one 256^3 box with 4 ghost zones,
periodic, gamma = 5/3, seeded smooth density wave rho = 1 + 0.1 sin(2 pi (x+y+z)),
velocity (1, 0.5, 0.25), p = 1 + 1e-3 U(-1,1).  One benchmark step is one full
hydro time step (ghost fill, dt reduction, primitive variables, flattening,
PPM + characteristic tracing, 12 HLLC solves per zone through the 3D CTU
corrections, flux-divergence update), replayed from the step's CUDA graph as
a user's hydro_step call runs it.  Metric: zone-updates/s = interior zones x
steps / device time.  The state (0.7 GB) and scratch (20 GB) are far larger
than L2, so no explicit flush is needed between steps.  Per-stage times come
from a separate profiled pass after the timed region.

The line also carries the other forms and configurations: mixed precision
on the same box, the Sod 32^3 box (single-box latency), 512 uneven Sedov
boxes (batched), the 512^3 Kelvin-Helmholtz box (largest single-GPU case, FP64
and mixed), the served request stream, and the method variants; each reports
zone-updates/s and p50/p99 latency.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank advances its own replica box (weak scaling, no
data-path collective: boxes are independent problems).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "zone-updates/s (FP64 & mixed <=1e-5 rel L1) + p50/p99 served-solve latency"
UNIT = "zone-updates/s"
N_BOX = 256

# Nominal pipe peaks, kept beside the measured ones the roofline divides by
# (hydro_measure_peaks runs a multiply-add probe on every SM in the same run):
# FP64 152 SMs x 4 flop/clk/SM x 2070 MHz = 1.26 TFLOP/s; FP32 152 SMs x 128
# lanes x 2 flop x 2070 MHz = 80.5 TFLOP/s.
FP64_NOMINAL_FLOPS = 152 * 4 * 2070e6
FP32_NOMINAL_FLOPS = 152 * 128 * 2 * 2070e6
# The stages the mixed form computes in FP32 (the rest stay FP64).
FP32_STAGES_MIXED = ("flatten", "slopes", "trace", "riemann", "ctu1", "ctu2")

# Algorithmic FP64 flops (add/sub, mul, div, sqrt; each counts 1) per unit of
# work of each stage, counted by the oracle (python -m oracle.count_flops
# density_wave 256: one step of this workload, every quantity formed once).
FLOPS_PER_UNIT = {
    "prim": 16.00, "flatten": 21.00, "slopes": 20.27, "trace": 320.58, "riemann": 125.00,
    "ctu1": 207.00, "ctu2": 237.00, "update": 55.00,
}


# DRAM bytes (read + write) per unit from one ncu capture of the kernel as it
# stands; a stage missing here has no capture of its current code and reports
# traffic null.
TRAFFIC_BYTES_PER_UNIT = {"ctu1": (19.339838e9 + 4.109397e9) / 101846016}  # k_ctu1<double, 0>, 256^3 capture: 23.45 GB / 101.8 M faces

# FP64-pipe warp-instruction slots per unit (x 32 lanes) from the same capture.
# With the products on the integer pipe, the FP64 pipe's ceiling for the
# kernel's own mix is its peak x (algorithmic flops per unit) / (2 x slots per
# unit): the rate at which the kernel would run with that pipe always busy.
FP64_SLOTS_PER_UNIT = {"ctu1": 83.0}


# Compulsory HBM traffic of one zone-update in every form: the FP64 state
# (5 doubles per zone) read and written once per step.
STATE_BYTES_PER_ZONE_UPDATE = 2 * 5 * 8


def hbm_peak_gbs():
    """The measured HBM copy bandwidth of these GPUs (GB/s) and where it comes from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, TypeError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


BOUND_FP64 = "the FP64 step is bound by the FP64 pipe (see roofline), so this is HBM headroom"
BOUND_MIXED = ("the mixed step is bound by its FP32 kernels' latency and issue rate and by the FP64 primitive "
               "conversion and update (see fp32_pipe), not by HBM")
BOUND_SERVED = "the served mix runs FP64 and mixed boxes; neither form is HBM-bound"


def hbm_fraction(zone_updates_per_s: float, bound: str = BOUND_FP64) -> dict:
    """A rate's compulsory state traffic as a fraction of the HBM roofline."""
    peak, src = hbm_peak_gbs()
    gbs = zone_updates_per_s * STATE_BYTES_PER_ZONE_UPDATE / 1e9
    return {"bytes_per_zone_update": STATE_BYTES_PER_ZONE_UPDATE, "achieved_gbs": gbs, "peak_gbs": peak,
            "frac": gbs / peak, "peak_source": src,
            "what": "compulsory traffic (the FP64 state read and written once per step) at the measured rate; "
                    + bound}


def fp32_pipe(n, step_ms: float, stage_ms: dict, peak_flops: float | None = None) -> dict:
    """Algorithmic flops of the mixed form's FP32 stages (the oracle's counts,
    which hold for either precision) per second, over the whole step and over
    those stages' own time, against the FP32 peak (measured when given)."""
    peak = peak_flops or FP32_NOMINAL_FLOPS
    flops = sum(FLOPS_PER_UNIT[s] * units_per_launch(s, n) for s in FP32_STAGES_MIXED)
    own_ms = sum(stage_ms.get(s, 0.0) for s in FP32_STAGES_MIXED)
    whole = flops / (step_ms * 1e-3)
    own = flops / (own_ms * 1e-3) if own_ms > 0 else None
    return {"algorithmic_tflops_whole_step": whole / 1e12, "frac_whole_step": whole / peak,
            "algorithmic_tflops_in_fp32_stages": None if own is None else own / 1e12,
            "frac_in_fp32_stages": None if own is None else own / peak,
            "peak_tflops": peak / 1e12,
            "peak_source": ("measured: FP32 multiply-add probe (hydro_measure_peaks), this run" if peak_flops
                            else "nominal: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"),
            "stages": list(FP32_STAGES_MIXED)}


def latency_stats(step_ms) -> dict:
    """p50/p99 of per-step device times (ms)."""
    import numpy as np
    a = np.asarray(step_ms, dtype=float)
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "max_ms": float(a.max()), "samples": int(a.size)}


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest of the ranks' values of x (x itself on one rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank: float, seconds: float, world: int, dist=None, device="cuda") -> float:
    """Units processed by all ranks per second of the slowest rank's time."""
    return world * units_per_rank / max_over_ranks(seconds, dist, device)


def units_per_launch(stage: str, n) -> int:
    """Units of work one launch of `stage` processes on a box of n = (nx, ny, nz)."""
    nx, ny, nz = n
    N = nx * ny * nz
    ext = (nx + 2) * (ny + 2) * (nz + 2)
    nn = (nx, ny, nz)
    if stage == "prim":
        return (nx + 8) * (ny + 8) * (nz + 8)
    if stage == "flatten":
        return ext
    if stage == "trace":
        return 3 * ext
    if stage == "slopes":
        return sum((nn[d] + 4) * (nn[(d + 1) % 3] + 2) * (nn[(d + 2) % 3] + 2) for d in range(3))
    if stage == "update":
        return N
    tot = 0
    for d in range(3):
        e, f = (d + 1) % 3, (d + 2) % 3
        if stage == "riemann":
            tot += (nn[d] + 1) * (nn[e] + 2) * (nn[f] + 2)
        elif stage == "ctu1":
            tot += (nn[d] + 1) * nn[e] * (nn[f] + 2) + (nn[d] + 1) * nn[f] * (nn[e] + 2)
        elif stage == "ctu2":
            tot += (nn[d] + 1) * nn[e] * nn[f]
    return tot


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ CPU oracle leg
def oracle_sample(seconds: float, n: int = 64, min_steps: int = 2, nthreads: int | None = None):
    """Times the oracle (as it stands) on a density-wave box of n^3 zones with the
    same recipe; returns (zone-updates/s, steps, threads)."""
    import oracle
    from paper_2007_05218_gb300 import inputs
    threads = nthreads or len(os.sched_getaffinity(0))
    pr = inputs.density_wave(n, seed=0)
    box = oracle.box_of(pr)
    Ug = oracle.embed(pr.U)
    steps, t0 = 0, time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < seconds:
        oracle.fill_ghosts(box, Ug)
        dt = oracle.compute_dt(box, Ug)
        rc, _ = oracle.step(box, Ug, dt, nthreads=threads)
        if rc:
            raise RuntimeError(f"oracle step failed: {rc}")
        steps += 1
    el = time.perf_counter() - t0
    return n ** 3 * steps / el, steps, threads


def oracle_rate(problems, steps: int, nthreads: int):
    """Times the oracle (as it stands) advancing every problem by `steps` steps
    (ghost fill, dt and update, box after box); returns (zone-updates/s, s)."""
    import oracle
    work = [(oracle.box_of(pr), oracle.embed(pr.U)) for pr in problems]
    zones = sum(int(pr.U[0].size) for pr in problems)
    t0 = time.perf_counter()
    for _ in range(steps):
        for box, Ug in work:
            oracle.fill_ghosts(box, Ug)
            dt = oracle.compute_dt(box, Ug)
            rc, _ = oracle.step(box, Ug, dt, nthreads=nthreads)
            if rc:
                raise RuntimeError(f"oracle step failed: {rc}")
    el = time.perf_counter() - t0
    return zones * steps / el, el


def oracle_configs(threads: int) -> dict:
    """The oracle on the other workloads, on all cores and on one thread: the
    Sod 32^3 box in full (20 steps), the first 32 boxes of the 512-box Sedov
    batch and a 128^3 box of the shear-layer recipe (2 steps each)."""
    from paper_2007_05218_gb300 import inputs
    cases = {"sod_32": ("Sod 32^3, the full 20 steps", lambda: [inputs.sod(32, axis=0, nsteps=20)], 20),
             "sedov_batch_512": ("the first 32 of the 512 Sedov boxes, 2 steps",
                                 lambda: inputs.sedov_batch(512, seed=0, nsteps=30)[:32], 2),
             "kelvin_helmholtz_512": ("a 128^3 box of the same shear-layer recipe, 2 steps",
                                      lambda: [inputs.kelvin_helmholtz(128, seed=0)], 2)}
    out = {}
    for name, (sample, make, steps) in cases.items():
        v, _ = oracle_rate(make(), steps, threads)
        v1, _ = oracle_rate(make(), steps, 1)
        out[name] = {"value": v, "cores": threads, "one_thread": v1, "unit": UNIT, "sample": sample}
    return out


def run_reference(args, rank: int) -> None:
    """Reference arm: the FP64 oracle on the host cores, on the benchmark's own
    256^3 density-wave box, one oracle step per benchmark step (a 2 s step on
    16 Grace cores; --box gives a smaller box for quick checks)."""
    if rank != 0:
        return
    import oracle
    from paper_2007_05218_gb300 import inputs
    threads = len(os.sched_getaffinity(0))
    n = args.box
    pr = inputs.density_wave(n, seed=0)
    box = oracle.box_of(pr)
    Ug = oracle.embed(pr.U)

    def one():
        oracle.fill_ghosts(box, Ug)
        dt = oracle.compute_dt(box, Ug)
        rc, _ = oracle.step(box, Ug, dt, nthreads=threads)
        if rc:
            raise RuntimeError(f"oracle step failed: {rc}")

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    value = n ** 3 * args.steps / el
    sample = (f"density wave {n}^3 (the benchmark's own box and recipe), {args.steps} oracle steps after "
              f"{args.warmup} warm-up steps, {threads} OpenMP threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": f"density_wave_{n}", "box": [n] * 3, "ghosts": 4,
                                        "gamma": 5.0 / 3.0, "bc": "periodic", "cfl": 0.5, "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------ timed helpers
def timed_steps(hydro, torch, h, nsteps, stream, dt_dev=None):
    """nsteps hydro_step calls on the step graph, one event between steps;
    returns (total ms, per-step ms)."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps + 1)]
    ev[0].record(stream)
    for k in range(nsteps):
        hydro.hydro_step(h, dt_dev, 1, stream)
        ev[k + 1].record(stream)
    ev[-1].synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(nsteps)]
    return ev[0].elapsed_time(ev[-1]), per


def stage_profile(hydro, torch, h, nsteps, stream):
    """Per-stage event times over nsteps profiled steps (launches bracketed by
    events, no graph): {stage: (kernels per step, ms per step)} and the
    profiled dict itself."""
    torch.cuda.synchronize()
    hydro.hydro_profile_begin(h)
    for _ in range(nsteps):
        hydro.hydro_step(h, None, 1, stream)
    torch.cuda.synchronize()
    prof = hydro.hydro_profile_end(h)
    return prof, {k: v[1] / nsteps for k, v in prof.items()}


# ------------------------------------------------------- batched uneven boxes
def run_batched(hydro, inputs, torch, np, stream, nboxes=512, nsteps=30):
    """512 independent Sedov boxes with edges drawn from {16,24,32,48,64}, 30
    steps in one handle (one launch per stage over all boxes, one CUDA graph
    per step), launch shapes autotuned first; FP64 and mixed precision."""
    probs = inputs.sedov_batch(nboxes, seed=0, nsteps=nsteps)
    zones = sum(p.zones for p in probs)
    out = {"workload": f"sedov_batch_{nboxes}", "boxes": nboxes, "zones": zones, "steps": nsteps}
    finals = {}
    for name, prec in (("fp64", hydro.HYDRO_FP64), ("mixed", hydro.HYDRO_MIXED)):
        B = hydro.Boxes(probs, precision=prec)
        tuned = hydro.hydro_autotune(B.h, reps=2, stream=stream)
        B.step(1)  # captures the step graph
        B.sync()
        for k, p in enumerate(probs):
            B.set_interior(k, p.U)
        torch.cuda.synchronize()
        ms, per = timed_steps(hydro, torch, B.h, nsteps, stream)
        B.sync()
        finals[name] = [B.interior(k)[[0, 4]] for k in range(nboxes)]
        B.close()
        del B
        rate = zones * nsteps / (ms * 1e-3)
        out[name] = {"value": rate, "unit": UNIT, "ms_per_step": ms / nsteps,
                     "step_latency": latency_stats(per),
                     "hbm": hbm_fraction(rate, BOUND_FP64 if name == "fp64" else BOUND_MIXED),
                     "tuned": {f"{t[0]}{'' if t[1] == 0 else '_mixed'}": [t[2], t[3]] for t in tuned}}
    worst = {n: max(float(np.abs(finals["mixed"][k][i] - finals["fp64"][k][i]).sum()
                          / np.abs(finals["fp64"][k][i]).sum()) for k in range(nboxes))
             for n, i in (("rho", 0), ("E", 1))}
    out["mixed"]["worst_box_rel_l1_vs_fp64"] = worst
    # the persistent form: all steps in one launch, per-box waits instead of
    # device-wide barriers between stages (128-thread blocks, not autotuned)
    for name, prec in (("fp64", hydro.HYDRO_FP64), ("mixed", hydro.HYDRO_MIXED)):
        P = hydro.Boxes(probs, precision=prec)
        hydro.hydro_persistent(P.h, True)
        P.step(1)
        P.sync()
        for k, p in enumerate(probs):
            P.set_interior(k, p.U)
        hydro.hydro_upload(P.h, np.concatenate([p.U.ravel() for p in probs]), stream)
        hydro.hydro_get_time(P.h, nboxes, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hydro.hydro_step(P.h, None, nsteps, stream)
        e1.record(stream)
        e1.synchronize()
        P.sync()
        ms = e0.elapsed_time(e1)
        same = all(np.array_equal(P.interior(k)[[0, 4]], finals[name][k]) for k in range(nboxes))
        P.close()
        del P
        rate = zones * nsteps / (ms * 1e-3)
        out[name]["persistent"] = {"value": rate, "unit": UNIT, "ms_per_step": ms / nsteps, "launches": 1,
                                   "bitwise_equal_to_per_stage_form": bool(same)}
    return out


# ------------------------------------------------------ Sod 32^3 (one box)
def run_sod(hydro, inputs, torch, np, stream, solves=20):
    """The Sod shock tube in one 32^3 box, 20 steps: per-step device latency on
    the step graph, and the whole solve through the C ABI (pinned host initial
    state -> 20 steps -> host result), repeated `solves` times."""
    pr = inputs.sod(32, axis=0, nsteps=20)
    B = hydro.Boxes([pr])
    B.step(3)
    B.sync()
    hydro.hydro_upload(B.h, pr.U, stream)
    torch.cuda.synchronize()
    ms, per = timed_steps(hydro, torch, B.h, pr.nsteps, stream)
    B.sync()
    host_in = torch.empty(pr.U.size, dtype=torch.float64, pin_memory=True)
    host_in.numpy()[:] = pr.U.ravel()
    host_out = torch.empty(pr.U.size, dtype=torch.float64, pin_memory=True)
    wall = []
    for _ in range(solves):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hydro.hydro_upload(B.h, host_in.numpy(), stream)
        hydro.hydro_step(B.h, None, pr.nsteps, stream)
        hydro.hydro_download(B.h, host_out.numpy(), stream)
        wall.append(time.perf_counter() - t0)
    B.sync()
    B.close()
    wall_ms = [1e3 * w for w in wall]
    return {"workload": "sod_32", "box": [32, 32, 32], "steps": pr.nsteps, "precision": "fp64",
            "value": pr.zones * pr.nsteps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / pr.nsteps,
            "step_latency": latency_stats(per),
            "solve_latency": {"p50_ms": float(np.percentile(wall_ms, 50)),
                              "p99_ms": float(np.percentile(wall_ms, 99)), "samples": solves,
                              "what": "host wall time of hydro_upload + 20 steps + hydro_download"}}


# ------------------------------------ Kelvin-Helmholtz 512^3 (largest box)
def run_kh512(hydro, inputs, torch, np, stream, fp64_steps, mixed_steps, n=512):
    """The 512^3 shear layer (periodic x, z; reflecting y), FP64 and mixed
    precision on the step graph.  The FP64 form is timed over fp64_steps steps
    (its rate per step does not depend on how many are run; 100 FP64 steps
    would hold the GPU for about a minute); the mixed form over mixed_steps;
    the relative L1 of mixed against FP64 is taken after the same fp64_steps
    steps from the same initial state."""
    pr = inputs.kelvin_helmholtz(n, seed=0)
    N = pr.zones
    out = {"workload": f"kelvin_helmholtz_{n}", "box": [n] * 3, "bc": "periodic x,z; reflect y"}
    res = {}
    for name, prec, nsteps in (("fp64", hydro.HYDRO_FP64, fp64_steps), ("mixed", hydro.HYDRO_MIXED, mixed_steps)):
        torch.cuda.empty_cache()
        B = hydro.Boxes([pr], precision=prec)
        gb = (B.state_bytes + B.scratch_bytes) / 1e9
        B.step(2)
        B.sync()
        hydro.hydro_upload(B.h, pr.U, stream)
        hydro.hydro_get_time(B.h, 1, stream)
        torch.cuda.synchronize()
        ms1, per1 = timed_steps(hydro, torch, B.h, fp64_steps, stream)
        B.sync()
        res[name] = B.interior(0)[[0, 4]]
        ms2, per2 = (0.0, [])
        if nsteps > fp64_steps:
            ms2, per2 = timed_steps(hydro, torch, B.h, nsteps - fp64_steps, stream)
            B.sync()
        B.close()
        del B
        torch.cuda.empty_cache()
        ms = ms1 + ms2
        rate = N * nsteps / (ms * 1e-3)
        out[name] = {"value": rate, "unit": UNIT, "steps": nsteps, "ms_per_step": ms / nsteps,
                     "step_latency": latency_stats(per1 + per2), "device_gb": gb,
                     "hbm": hbm_fraction(rate, BOUND_FP64 if name == "fp64" else BOUND_MIXED)}
    out["mixed"]["rel_l1_vs_fp64"] = {
        "after_steps": fp64_steps,
        "rho": float(np.abs(res["mixed"][0] - res["fp64"][0]).sum() / np.abs(res["fp64"][0]).sum()),
        "E": float(np.abs(res["mixed"][1] - res["fp64"][1]).sum() / np.abs(res["fp64"][1]).sum())}
    return out


# ------------------------------------------------------------ method variants
def run_variants(hydro, torch, pr, stream, warmup, nsteps=20):
    """The method variants on the same box, FP64: Colella-Sekora limiter,
    two-shock Riemann solver, both.  W warm-up steps, nsteps timed on the step
    graph, then a short profiled pass for the stage times."""
    out = {}
    N = pr.U[0].size
    for name, lim, rs in (("cs08", hydro.HYDRO_LIMITER_CS08, hydro.HYDRO_RIEMANN_HLLC),
                          ("two_shock", hydro.HYDRO_LIMITER_CW84, hydro.HYDRO_RIEMANN_TWO_SHOCK),
                          ("cs08_two_shock", hydro.HYDRO_LIMITER_CS08, hydro.HYDRO_RIEMANN_TWO_SHOCK)):
        V = hydro.Boxes([pr], limiter=lim, riemann=rs)
        V.step(warmup)
        V.sync()
        torch.cuda.synchronize()
        ms, per = timed_steps(hydro, torch, V.h, nsteps, stream)
        _, stages = stage_profile(hydro, torch, V.h, 3, stream)
        V.sync()
        V.close()
        out[name] = {"value": N * nsteps / (ms * 1e-3), "unit": UNIT, "steps": nsteps,
                     "ms_per_step": ms / nsteps, "step_latency": latency_stats(per),
                     "stages_ms_per_step": stages}
    return out


# ------------------------------------------------------------ served stream
def run_served(hydro, inputs, torch, np, nrequests, rate=200.0, budget_gb=120.0, max_active=256):
    """Continuous batching of a seeded request stream (Poisson arrivals at
    `rate`/s, box edges uniform in [32,128], 10-200 steps, Sod/Sedov/shear-layer
    initial states, FP64 or mixed with equal odds) under a device memory
    budget; requests are submitted at their arrival times through
    hydro_submit and collected with hydro_poll."""
    import time as _t
    stream = inputs.served_stream(nrequests, seed=0, rate_per_s=rate)
    work = sum(r.problem.zones * r.nsteps for r in stream)
    torch.cuda.empty_cache()
    srv = hydro.Server(int(budget_gb * 1e9), max_active=max_active)
    outs = [np.zeros((5,) + r.problem.U.shape[1:]) for r in stream]
    pending = {}
    lat, queued = [], []
    t0 = _t.perf_counter()
    k = 0
    while k < len(stream) or pending:
        now = _t.perf_counter() - t0
        while k < len(stream) and stream[k].arrival_s <= now:
            r = stream[k]
            prec = hydro.HYDRO_MIXED if r.mixed else hydro.HYDRO_FP64
            pending[srv.submit(r.problem, nsteps=r.nsteps, precision=prec)] = k
            k += 1
        for t in list(pending):
            rc, info = hydro.hydro_poll(srv.s, t, outs[pending[t]])
            if rc == hydro.HYDRO_PENDING:
                continue
            if rc != hydro.HYDRO_OK:
                raise RuntimeError(f"served request {pending[t]} failed: {rc}")
            lat.append(info.latency_s)
            queued.append(info.queued_s)
            del pending[t]
        _t.sleep(0.0002)
    makespan = _t.perf_counter() - t0
    st = srv.stats()
    srv.close()
    del srv
    torch.cuda.empty_cache()
    span_arrivals = stream[-1].arrival_s
    return {"workload": f"served_stream_{nrequests}", "requests": nrequests,
            "offered_rate_req_per_s": rate,
            "offered_zone_updates_per_s": work / span_arrivals if span_arrivals > 0 else None,
            "value": work / makespan, "unit": UNIT, "hbm": hbm_fraction(work / makespan, BOUND_SERVED),
            "makespan_s": makespan, "arrival_span_s": span_arrivals,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_queued_s": float(np.mean(queued)), "p99_queued_s": float(np.percentile(queued, 99)),
            "budget_gb": budget_gb, "max_active": max_active,
            "peak_pool_gb": st["peak_bytes"] / 1e9, "ticks": st["ticks"],
            "kernel_launches": st["kernel_launches"],
            "mix": {"mixed": sum(r.mixed for r in stream),
                    "sod": sum(r.problem.name == "sod" for r in stream),
                    "sedov": sum(r.problem.name == "sedov" for r in stream),
                    "kelvin_helmholtz": sum(r.problem.name == "kelvin_helmholtz" for r in stream)}}


# ------------------------------------------------------------------ main arm
def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-box batched measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the limiter / Riemann variant measurement")
    ap.add_argument("--no-sod", action="store_true", help="skip the Sod 32^3 latency measurement")
    ap.add_argument("--no-kh512", action="store_true", help="skip the 512^3 shear-layer measurement")
    ap.add_argument("--kh512-fp64-steps", type=int, default=10)
    ap.add_argument("--kh512-mixed-steps", type=int, default=100)
    ap.add_argument("--served-requests", type=int, default=48,
                    help="length of the served request stream (0 skips it; the full stream is 2000)")
    ap.add_argument("--served-rate", type=float, default=200.0, help="mean arrival rate of the served stream (1/s)")
    ap.add_argument("--only-served", action="store_true", help="run the served stream alone and print its record")
    ap.add_argument("--box", type=int, default=N_BOX, help="box edge (default 256; smaller only for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    from paper_2007_05218_gb300 import hydro, inputs

    torch.cuda.set_device(local)
    if args.only_served:
        print(json.dumps(run_served(hydro, inputs, torch, np, args.served_requests, args.served_rate)), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()
    peaks = hydro.hydro_measure_peaks(stream)

    nb = args.box
    n = (nb, nb, nb)
    N = nb ** 3
    pr = inputs.density_wave(nb, seed=rank)
    B = hydro.Boxes([pr])
    B_state_gb, B_scratch_gb = B.state_bytes / 1e9, B.scratch_bytes / 1e9
    B.step(args.warmup)  # the first call captures the step graph
    B.sync()

    # ---- device-timed region: K steps replayed from the step graph, as hydro_step runs them
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    launches0 = hydro.hydro_kernel_launches(B.h)
    ms, per_step = timed_steps(hydro, torch, B.h, args.steps, stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = hydro.hydro_kernel_launches(B.h) - launches0
    B.sync()  # raises on a nonphysical state
    ms_max = max_over_ranks(ms, dist)
    value = whole_job_rate(N * args.steps, ms_max * 1e-3, world)  # ms_max: the slowest rank's time already
    # ---- per-stage times: a separate profiled pass (events around every stage launch)
    prof, stages_ms = stage_profile(hydro, torch, B.h, min(args.steps, 5), stream)
    nprof = min(args.steps, 5)

    # ---- end to end through the C ABI: pinned host IC -> K steps -> host result
    nbytes = pr.U.nbytes
    host_in = torch.empty(pr.U.size, dtype=torch.float64, pin_memory=True)
    host_in.numpy()[:] = pr.U.ravel()
    host_out = torch.empty(pr.U.size, dtype=torch.float64, pin_memory=True)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hydro.hydro_upload(B.h, host_in.numpy(), stream)
    hydro.hydro_step(B.h, None, args.steps, stream)
    hydro.hydro_download(B.h, host_out.numpy(), stream)
    e2e_s = time.perf_counter() - t0
    B.sync()
    e2e = {"value": whole_job_rate(N * args.steps, e2e_s, world, dist), "unit": UNIT,
           "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": nbytes / args.steps,
           "what": "hydro_upload of the interior initial state from pinned host memory, K steps, "
                   "hydro_download of the final interior state (bytes per step = solve bytes / K)"}
    B.close()
    del B
    fp64_final = host_out.numpy().reshape(pr.U.shape)

    # ---- mixed precision on the same workload: W warm-up steps, re-upload the
    # initial state, K timed steps; accuracy against the FP64 result after the
    # same K steps from the same initial state
    M = hydro.Boxes([pr], precision=hydro.HYDRO_MIXED)
    M.step(args.warmup)
    M.sync()
    hydro.hydro_upload(M.h, host_in.numpy(), stream)
    hydro.hydro_get_time(M.h, 1, stream)
    barrier()
    torch.cuda.synchronize()
    ms_mixed, per_mixed = timed_steps(hydro, torch, M.h, args.steps, stream)
    M.sync()
    mixed_final = np.zeros_like(fp64_final)
    hydro.hydro_download(M.h, mixed_final, stream)
    _, mixed_stage_ms = stage_profile(hydro, torch, M.h, nprof, stream)
    M.close()
    del M
    rel_l1 = {name: float(np.abs(mixed_final[v] - fp64_final[v]).sum() / np.abs(fp64_final[v]).sum())
              for name, v in (("rho", 0), ("E", 4))}
    # the same with the fused tile stage (tile shape and z-segment autotuned)
    Mt = hydro.Boxes([pr], precision=hydro.HYDRO_MIXED)
    hydro.hydro_fuse_tiles(Mt.h, True)
    tile_tuned = [t for t in hydro.hydro_autotune(Mt.h, reps=2, stream=stream) if t[0] == "tile"]
    Mt.step(args.warmup)
    Mt.sync()
    hydro.hydro_upload(Mt.h, host_in.numpy(), stream)
    hydro.hydro_get_time(Mt.h, 1, stream)
    torch.cuda.synchronize()
    ms_tile, per_tile = timed_steps(hydro, torch, Mt.h, args.steps, stream)
    Mt.sync()
    tile_final = np.zeros_like(fp64_final)
    hydro.hydro_download(Mt.h, tile_final, stream)
    _, tile_stage_ms = stage_profile(hydro, torch, Mt.h, nprof, stream)
    Mt.close()
    del Mt
    tile_rate = whole_job_rate(N * args.steps, ms_tile * 1e-3, world, dist)
    mixed_tile = {"value": tile_rate, "unit": UNIT, "ms_per_step": ms_tile / args.steps,
                  "step_latency": latency_stats(per_tile), "hbm": hbm_fraction(tile_rate, BOUND_MIXED),
                  "bitwise_equal_to_line_stage": bool(np.array_equal(tile_final, mixed_final)),
                  "tile": {"rows": tile_tuned[0][5], "seg": tile_tuned[0][6], "order": tile_tuned[0][3]}
                  if tile_tuned else None,
                  "stages_ms_per_step": tile_stage_ms}
    mixed_rate = whole_job_rate(N * args.steps, ms_mixed * 1e-3, world, dist)
    mixed = {"value": mixed_rate, "unit": UNIT, "hbm": hbm_fraction(mixed_rate, BOUND_MIXED),
             "fp32_pipe": fp32_pipe(n, ms_mixed / args.steps, mixed_stage_ms, peaks["fp32_flops"]),
             "ms_per_step": ms_mixed / args.steps, "step_latency": latency_stats(per_mixed),
             "dtype": "f32 reconstruct/trace/Riemann, f64 state/update/dt",
             "rel_l1_vs_fp64": rel_l1, "stages_ms_per_step": mixed_stage_ms, "fused_tile": mixed_tile}
    sod = None if args.no_sod else run_sod(hydro, inputs, torch, np, stream)
    variants = None if args.no_variants else run_variants(hydro, torch, pr, stream, args.warmup)
    batched = None if args.no_batched else run_batched(hydro, inputs, torch, np, stream)
    kh512 = None if args.no_kh512 else run_kh512(hydro, inputs, torch, np, stream, args.kh512_fp64_steps,
                                                 args.kh512_mixed_steps)
    served = (run_served(hydro, inputs, torch, np, args.served_requests, args.served_rate)
              if args.served_requests > 0 else None)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel: algorithmic flops per launch over
    # its average launch time in the profiled pass, against the measured FP64
    # multiply-add rate of this GPU
    stage_l = {k: v for k, v in prof.items() if k in FLOPS_PER_UNIT}
    top = max(stage_l, key=lambda k: stage_l[k][1])
    nlaunch, tot_ms = stage_l[top]
    avg_s = tot_ms / nlaunch * 1e-3
    flops = FLOPS_PER_UNIT[top] * units_per_launch(top, n)
    achieved = flops / avg_s
    fp64_probe = peaks["fp64_flops"]
    roofline = {"bound": "alu", "kernel": f"k_{top}", "achieved": achieved / 1e12,
                "peak": FP64_NOMINAL_FLOPS / 1e12, "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_FLOPS,
                "traffic": (TRAFFIC_BYTES_PER_UNIT[top] * units_per_launch(top, n)
                            if top in TRAFFIC_BYTES_PER_UNIT else None),
                "peak_source": "derived from unit counts and clocks: 152 SMs x 4 FP64 flop/clk/SM x 2070 MHz",
                "note": ("the kernel forms its FP64 products (45 of the 128 FP64 operations of a corrected face) "
                         "on the integer pipe, bitwise the FP64 multiply; achieved counts all of its algorithmic "
                         "flops against the FP64 pipe's peak, so frac can pass what that pipe alone delivers; "
                         "mix_ceiling is that pipe's peak for the kernel's own FP64 instruction mix"),
                "mix_ceiling": (FP64_NOMINAL_FLOPS * FLOPS_PER_UNIT[top] / (2.0 * FP64_SLOTS_PER_UNIT[top]) / 1e12
                                if top in FP64_SLOTS_PER_UNIT else None),
                "frac_of_mix_ceiling": (achieved / (FP64_NOMINAL_FLOPS * FLOPS_PER_UNIT[top] / (2.0 * FP64_SLOTS_PER_UNIT[top]))
                                        if top in FP64_SLOTS_PER_UNIT else None),
                "fp64_slots_per_unit": FP64_SLOTS_PER_UNIT.get(top),
                "peak_measured": fp64_probe / 1e12, "frac_of_measured": achieved / fp64_probe,
                "peak_measured_source": "FP64 multiply-add probe on every SM (hydro_measure_peaks), this run",
                "kernel_time_source": f"events around each stage launch, {nprof} profiled steps after the timed region",
                "flops_per_launch": flops}
    hbm = hbm_fraction(value, BOUND_FP64)
    if roofline["traffic"] is not None:
        # the dominant kernel's DRAM bytes per launch (ncu) over its live launch time
        gbs = roofline["traffic"] / avg_s / 1e9
        hbm["dominant_kernel"] = {"kernel": f"k_{top}", "dram_gbs": gbs, "frac": gbs / hbm["peak_gbs"]}
    total_flops = sum(FLOPS_PER_UNIT[s] * units_per_launch(s, n) for s in FLOPS_PER_UNIT)
    step_fp64 = total_flops / (ms / args.steps * 1e-3)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, steps, threads = oracle_sample(10.0)
        v1, steps1, _ = oracle_sample(10.0, n=32, nthreads=1)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"density wave 64^3 (same recipe), {steps} oracle steps on {threads} threads",
               "one_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"density wave 32^3 (same recipe), {steps1} oracle steps on 1 thread"},
               "configs": oracle_configs(threads)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"density_wave_{nb}", "box": list(n), "ghosts": 4, "gamma": 5.0 / 3.0,
                   "bc": "periodic", "cfl": 0.5, "precision": "fp64",
                   "l2": "inputs larger than L2 (state %.1f GB + scratch %.1f GB per box)"
                         % (B_state_gb, B_scratch_gb),
                   "timed_path": "hydro_step replaying the step's CUDA graph, profiling off",
                   "parallelism": f"replicas x{world}"},
        "step_latency": latency_stats(per_step),
        "roofline": roofline,
        "hbm": hbm,
        "peaks_measured": {"fp64_tflops": peaks["fp64_flops"] / 1e12, "fp32_tflops": peaks["fp32_flops"] / 1e12,
                           "sms": peaks["sms"]},
        "fp64_algorithmic_tflops_whole_step": step_fp64 / 1e12,
        "stages_ms_per_step": stages_ms,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "mixed": mixed,
        "sod_32": sod,
        "kelvin_helmholtz_512": kh512,
        "batched": batched,
        "served": served,
        "variants": variants,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
