#!/usr/bin/env python3
"""Benchmark: FP64 unsplit PPM/CTU/HLLC hydro update on one GB300.

Workload (the metric's FP64 configuration): one 256^3 box with 4 ghost zones,
periodic, gamma = 5/3, seeded smooth density wave rho = 1 + 0.1 sin(2 pi (x+y+z)),
velocity (1, 0.5, 0.25), p = 1 + 1e-3 U(-1,1).  One benchmark step is one full
hydro time step (ghost fill, dt reduction, primitive variables, flattening,
PPM + characteristic tracing, 12 HLLC solves per zone through the 3D CTU
corrections, flux-divergence update).  Metric: zone-updates/s = interior
zones x steps / device time.  The state (0.7 GB) and scratch (14 GB) are far
larger than L2, so no explicit flush is needed between steps.

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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "zone-updates/s (FP64 & mixed <=1e-5 rel L1) + p50/p99 served-solve latency"
UNIT = "zone-updates/s"
N_BOX = 256

# FP64 peak for the ALU roofline: 152 SMs x 4 FP64 flop/clk/SM x 2070 MHz.
# (GB300 nominal FP64 is 1.25 TFLOP/s; 1.25e12 / (152 x 2.07e9) = 4 flop/clk/SM.)
FP64_PEAK_FLOPS = 152 * 4 * 2070e6
# FP32 peak for the mixed form's FP32 stages: 152 SMs x 128 FP32 lanes x 2
# flop (fused multiply-add) x 2070 MHz = 80.5 TFLOP/s, nominal.
FP32_PEAK_FLOPS = 152 * 128 * 2 * 2070e6
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
TRAFFIC_BYTES_PER_UNIT = {"ctu1": (1.554235e9 + 0.519544e9) / 12879360}  # k_ctu1<double, 0>, 128^3 capture: 2.074 GB / 12.88 M faces


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


def hbm_fraction(zone_updates_per_s: float) -> dict:
    """A rate's compulsory state traffic as a fraction of the HBM roofline."""
    peak, src = hbm_peak_gbs()
    gbs = zone_updates_per_s * STATE_BYTES_PER_ZONE_UPDATE / 1e9
    return {"bytes_per_zone_update": STATE_BYTES_PER_ZONE_UPDATE, "achieved_gbs": gbs, "peak_gbs": peak,
            "frac": gbs / peak, "peak_source": src,
            "what": "compulsory traffic (the FP64 state read and written once per step) at the measured rate; "
                    "the step is bound by the FP64 pipe (see roofline), so this is the HBM headroom"}


def fp32_pipe(n, step_ms: float, stage_ms: dict) -> dict:
    """Algorithmic flops of the mixed form's FP32 stages (the oracle's counts,
    which hold for either precision) per second, over the whole step and over
    those stages' own time, against the FP32 peak."""
    flops = sum(FLOPS_PER_UNIT[s] * units_per_launch(s, n) for s in FP32_STAGES_MIXED)
    own_ms = sum(stage_ms.get(s, 0.0) for s in FP32_STAGES_MIXED)
    whole = flops / (step_ms * 1e-3)
    own = flops / (own_ms * 1e-3) if own_ms > 0 else None
    return {"algorithmic_tflops_whole_step": whole / 1e12, "frac_whole_step": whole / FP32_PEAK_FLOPS,
            "algorithmic_tflops_in_fp32_stages": None if own is None else own / 1e12,
            "frac_in_fp32_stages": None if own is None else own / FP32_PEAK_FLOPS,
            "peak_tflops": FP32_PEAK_FLOPS / 1e12,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (nominal)",
            "stages": list(FP32_STAGES_MIXED)}


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


def run_reference(args, rank: int) -> None:
    """Reference arm: the FP64 oracle on the host cores, one 64^3 density-wave
    step (same recipe) per benchmark step."""
    if rank != 0:
        return
    import oracle
    from paper_2007_05218_gb300 import inputs
    threads = len(os.sched_getaffinity(0))
    n = 64
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
    sample = f"density wave {n}^3 (same recipe as the 256^3 workload), one oracle step per benchmark step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": f"density_wave_{N_BOX}", "box": [N_BOX] * 3, "ghosts": 4,
                                        "gamma": 5.0 / 3.0, "bc": "periodic", "cfl": 0.5, "precision": "fp64",
                                        "sampled_as": f"{n}^3 box of the same recipe per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


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
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hydro.hydro_step(B.h, None, nsteps, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        B.sync()
        ms = e0.elapsed_time(e1)
        finals[name] = [B.interior(k)[[0, 4]] for k in range(nboxes)]
        B.close()
        del B
        rate = zones * nsteps / (ms * 1e-3)
        out[name] = {"value": rate, "unit": UNIT, "ms_per_step": ms / nsteps, "hbm": hbm_fraction(rate),
                     "tuned": {f"{t[0]}{'' if t[1] == 0 else '_mixed'}": [t[2], t[3]] for t in tuned}}
    worst = {n: max(float(np.abs(finals["mixed"][k][i] - finals["fp64"][k][i]).sum()
                          / np.abs(finals["fp64"][k][i]).sum()) for k in range(nboxes))
             for n, i in (("rho", 0), ("E", 1))}
    out["mixed"]["worst_box_rel_l1_vs_fp64"] = worst
    return out


# ------------------------------------------------------------ served stream
def run_variants(hydro, torch, pr, stream, warmup, nsteps=20):
    """The method variants on the same box, FP64: Colella-Sekora limiter,
    two-shock Riemann solver, both.  W warm-up steps, then nsteps timed with
    events on the launching stream; per-stage event times per step."""
    out = {}
    N = pr.U[0].size
    for name, lim, rs in (("cs08", hydro.HYDRO_LIMITER_CS08, hydro.HYDRO_RIEMANN_HLLC),
                          ("two_shock", hydro.HYDRO_LIMITER_CW84, hydro.HYDRO_RIEMANN_TWO_SHOCK),
                          ("cs08_two_shock", hydro.HYDRO_LIMITER_CS08, hydro.HYDRO_RIEMANN_TWO_SHOCK)):
        V = hydro.Boxes([pr], limiter=lim, riemann=rs)
        V.step(warmup)
        V.sync()
        torch.cuda.synchronize()
        hydro.hydro_profile_begin(V.h)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nsteps):
            hydro.hydro_step(V.h, None, 1, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        prof = hydro.hydro_profile_end(V.h)
        V.sync()
        V.close()
        out[name] = {"value": N * nsteps / (ms * 1e-3), "unit": UNIT, "steps": nsteps,
                     "ms_per_step": ms / nsteps,
                     "stages_ms_per_step": {k: v[1] / nsteps for k, v in prof.items()}}
    return out


def run_served(hydro, inputs, torch, np, nrequests, budget_gb=120.0, max_active=256):
    """Continuous batching of a seeded request stream (Poisson arrivals at
    200/s, box edges uniform in [32,128], 10-200 steps, Sod/Sedov/shear-layer
    initial states, FP64 or mixed with equal odds) under a device memory
    budget; requests are submitted at their arrival times through
    hydro_submit and collected with hydro_poll."""
    import time as _t
    stream = inputs.served_stream(nrequests, seed=0)
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
            "offered_rate_req_per_s": 200.0,
            "offered_zone_updates_per_s": work / span_arrivals if span_arrivals > 0 else None,
            "value": work / makespan, "unit": UNIT, "hbm": hbm_fraction(work / makespan), "makespan_s": makespan,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_queued_s": float(np.mean(queued)), "budget_gb": budget_gb, "max_active": max_active,
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
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-box batched measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the limiter / Riemann variant measurement")
    ap.add_argument("--served-requests", type=int, default=48,
                    help="length of the served request stream (0 skips it; the full stream is 2000)")
    ap.add_argument("--box", type=int, default=N_BOX, help="box edge (default 256; smaller only for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    from paper_2007_05218_gb300 import hydro, inputs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    nb = args.box
    n = (nb, nb, nb)
    N = nb ** 3
    pr = inputs.density_wave(nb, seed=rank)
    B = hydro.Boxes([pr])
    B_state_gb, B_scratch_gb = B.state_bytes / 1e9, B.scratch_bytes / 1e9
    stream = torch.cuda.current_stream()
    B.step(args.warmup)
    B.sync()

    # ---- device-timed region: K steps
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    launches0 = hydro.hydro_kernel_launches(B.h)
    hydro.hydro_profile_begin(B.h)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        hydro.hydro_step(B.h, None, 1, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = hydro.hydro_profile_end(B.h)
    launches = hydro.hydro_kernel_launches(B.h) - launches0
    B.sync()  # raises on a nonphysical state
    ms_max = max_over_ranks(ms, dist)
    value = whole_job_rate(N * args.steps, ms_max * 1e-3, world)  # ms_max: the slowest rank's time already

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
    hydro.hydro_profile_begin(M.h)
    e0.record(stream)
    for _ in range(args.steps):
        hydro.hydro_step(M.h, None, 1, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_mixed = e0.elapsed_time(e1)
    prof_mixed = hydro.hydro_profile_end(M.h)
    M.sync()
    mixed_final = np.zeros_like(fp64_final)
    hydro.hydro_download(M.h, mixed_final, stream)
    M.close()
    del M
    rel_l1 = {name: float(np.abs(mixed_final[v] - fp64_final[v]).sum() / np.abs(fp64_final[v]).sum())
              for name, v in (("rho", 0), ("E", 4))}
    variants = None if args.no_variants else run_variants(hydro, torch, pr, stream, args.warmup)
    batched = None if args.no_batched else run_batched(hydro, inputs, torch, np, stream)
    served = run_served(hydro, inputs, torch, np, args.served_requests) if args.served_requests > 0 else None
    mixed_rate = whole_job_rate(N * args.steps, ms_mixed * 1e-3, world, dist)
    mixed_stage_ms = {k: v[1] / args.steps for k, v in prof_mixed.items()}
    mixed = {"value": mixed_rate, "unit": UNIT, "hbm": hbm_fraction(mixed_rate),
             "fp32_pipe": fp32_pipe(n, ms_mixed / args.steps, mixed_stage_ms),
             "ms_per_step": ms_mixed / args.steps, "dtype": "f32 reconstruct/trace/Riemann, f64 state/update/dt",
             "rel_l1_vs_fp64": rel_l1, "stages_ms_per_step": mixed_stage_ms}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (live event times of this run)
    stage_ms = {k: v for k, v in prof.items() if k in FLOPS_PER_UNIT}
    top = max(stage_ms, key=lambda k: stage_ms[k][1])
    nlaunch, tot_ms = stage_ms[top]
    avg_s = tot_ms / nlaunch * 1e-3
    flops = FLOPS_PER_UNIT[top] * units_per_launch(top, n)
    achieved = flops / avg_s
    roofline = {"bound": "alu", "kernel": f"k_{top}", "achieved": achieved / 1e12, "peak": FP64_PEAK_FLOPS / 1e12,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_FLOPS,
                "traffic": (TRAFFIC_BYTES_PER_UNIT[top] * units_per_launch(top, n)
                            if top in TRAFFIC_BYTES_PER_UNIT else None),
                "peak_source": "derived: 152 SMs x 4 FP64 flop/clk/SM x 2070 MHz (nominal 1.25 TFLOP/s)",
                "flops_per_launch": flops}
    hbm = hbm_fraction(value)
    if roofline["traffic"] is not None:
        # the dominant kernel's DRAM bytes per launch (ncu) over its live launch time
        gbs = roofline["traffic"] / avg_s / 1e9
        hbm["dominant_kernel"] = {"kernel": f"k_{top}", "dram_gbs": gbs, "frac": gbs / hbm["peak_gbs"]}
    total_flops = sum(FLOPS_PER_UNIT[s] * units_per_launch(s, n) for s in FLOPS_PER_UNIT)
    step_fp64 = total_flops / (ms / args.steps * 1e-3)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, steps, threads = oracle_sample(10.0)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"density wave 64^3 (same recipe), {steps} oracle steps on {threads} threads"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"density_wave_{nb}", "box": list(n), "ghosts": 4, "gamma": 5.0 / 3.0,
                   "bc": "periodic", "cfl": 0.5, "precision": "fp64",
                   "l2": "inputs larger than L2 (state %.1f GB + scratch %.1f GB per box)"
                         % (B_state_gb, B_scratch_gb),
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "hbm": hbm,
        "fp64_algorithmic_tflops_whole_step": step_fp64 / 1e12,
        "stages_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "mixed": mixed,
        "variants": variants,
        "batched": batched,
        "served": served,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
