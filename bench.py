"""Throughput of the Enskog-Vlasov lattice Boltzmann step on GB300.

Workload (N = 1, per GPU): the 2-D static-droplet Laplace sweep -- nine
independent 1024 x 1024 periodic D2Q9 layers (T/Tc in {0.7, 0.8, 0.9} x droplet
radius in {64, 128, 256}, tanh interface of width 4, u = 0), thermal double
population, FP32 storage and arithmetic, Carnahan-Starling Enskog pressure with
b = 4, a = 0.1, kappa = 0.116 (10-90 % width 4 at T/Tc = 0.7), bare tau = 0.3, lambda = 1.  One step = one
lattice update of all nine layers (9 x 2^20 lattice updates).  The populations
(1.36 GB per step read + written) exceed the 129 MB L2, so no flush is needed.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead (the
reference arm), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 1024
TRS = (0.7, 0.8, 0.9)
RADII = (64.0, 128.0, 256.0)
A, B, KAPPA, TAU = 0.1, 4.0, 0.116, 0.3
# The ensemble's capillarity: kappa = 0.2 (10-90 % width 5.3 at T/Tc = 0.7, 9.6 at 0.9), as
# the surrogate workload; at 0.116 26 of the 512 domains diverge within 5000 steps, at 0.2 nine
# (coalescing pairs at T/Tc ~ 0.70, which the FP64 oracle does not hold either).
ENSEMBLE_KAPPA = 0.2
ENSEMBLE_STEPS = 5000
BYTES_PER_LU = 2 * 9 * 2 * 4          # D2Q9, f and g, read + write, FP32
# dram__bytes_read.sum + dram__bytes_write.sum of one launch on this workload, per launch
# shape (W, H) of the fused kernel (H = -1: the balanced grid, k_fused2d_bal), from one ncu
# capture each (profiles/fused2d_d2q9_thermal_fp32.md); a shape without a capture, or a
# changed kernel, reports None.
MEASURED_TRAFFIC_BYTES = {(128, 256): 1.3342e9, (128, -1): 1.3384e9}
# Floating-point operations per lattice update of the FP64 oracle's plain form of the
# step (every stencil and equilibrium product summed over all Q velocities), counted by
# running the oracle's source with a counting number type; tests/test_oracle_flops.py
# checks these values against that count.
ORACLE_FLOPS_PER_LU = {"d2q9_thermal": 2383, "d3q27_thermal": 10297}
# FP32 (non-tensor) peak: 152 SMs x 128 FP32 lanes x 2 operations (FMA) x SM clock.
FP32_LANES = 152 * 128
# DRAM bytes (read + write) of one step of the 512-domain ensemble per work-item shape,
# from one ncu capture of a one-step launch of k_batch (5.949 GB algorithmic;
# profiles/batch_ensemble_d2q9_fp32.md); None for other shapes or when the kernel changes.
ENSEMBLE_TRAFFIC_BYTES_PER_STEP = {(128, 256): 6.0400e9, (128, 512): 6.0011e9}
WORKLOAD = "droplet Laplace sweep: 9 x 1024^2 D2Q9 thermal, FP32"


def workload_fields(coexistence, critical_point, layers=None):
    """Initial fields of the sweep (rho, u, T) stacked along z."""
    from paper_2508_00577_gb300 import inputs
    _, Tc = critical_point(1, A, B)
    cases = []
    for tr in TRS:
        rv, rl = coexistence(1, A, B, tr * Tc)
        for R in RADII:
            cases.append((R, rv, rl, tr * Tc))
    if layers is not None:
        cases = [cases[k] for k in layers]
    return inputs.droplet_stack(NX, NY, cases), len(cases)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"evlbm_clocks_{os.getpid()}.csv")
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            try:
                with open(self.path) as fh:
                    self.lines = [l for l in fh.read().splitlines() if l.strip()]
                os.remove(self.path)
            except OSError:
                self.lines = []

    def summary(self):
        sm, mx, reasons = [], [], set()
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(self.NAMES, parts[2:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def emit(line, args):
    """Print the result line and, with --log, append it to a JSON-lines file."""
    text = json.dumps(line)
    print(text, flush=True)
    if getattr(args, "log", None):
        with open(args.log, "a") as fh:
            fh.write(text + "\n")


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, device=None):
    """The maximum of a per-rank number over all ranks (the job's time is the
    slowest rank's); the value itself when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, nodes_per_rank, steps, total_ms):
    """Whole-job throughput of `world` replicas, each updating nodes_per_rank nodes
    per step, timed by the slowest rank."""
    return world * nodes_per_rank * steps / (total_ms * 1e-3) / 1e6


def cpu_baseline(steps=None, budget_s=15.0):
    """The FP64 oracle on one 1024^2 layer of the workload (T/Tc = 0.8, R = 128)."""
    import oracle
    import oracle.eos as E
    (rho, u, T), _ = workload_fields(E.maxwell, E.critical_point, layers=[4])
    p = oracle.Params(Q=9, nx=NX, ny=NY, nz=1, eos=1, a=A, b=B, kappa=KAPPA, tau=TAU, thermal=1)
    s = oracle.State(p, rho, u, T)
    s.step(1)                                    # warm-up (page in, thread pool)
    t0 = time.perf_counter()
    n = 0
    while True:
        s.step(1)
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and el >= budget_s):
            break
    mlups = NX * NY * n / el / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one 1024^2 layer (T/Tc=0.8, R=128) of the sweep, {n} steps, {el:.1f} s"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import oracle.eos as E
    (rho, u, T), _ = workload_fields(E.maxwell, E.critical_point, layers=[4])
    p = oracle.Params(Q=9, nx=NX, ny=NY, nz=1, eos=1, a=A, b=B, kappa=KAPPA, tau=TAU, thermal=1)
    s = oracle.State(p, rho, u, T)
    for _ in range(args.warmup):
        s.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(1)
    el = time.perf_counter() - t0
    mlups = NX * NY * args.steps / el / 1e6
    sample = f"one 1024^2 layer (T/Tc=0.8, R=128) of the sweep per step, {args.steps} steps"
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line, args)
    return 0


def alu_check(mlups, flops_per_lu, sm_max_mhz=None):
    """Where the step would sit against the FP32 ALU roof if the kernel executed the
    oracle's plain arithmetic: its operation count at the measured update rate, against
    152 SMs x 128 lanes x 2 x the highest SM clock seen in the timed region (2070 MHz,
    the GB300's maximum, when no clock was sampled)."""
    mhz = sm_max_mhz or 2070.0
    peak = 2 * FP32_LANES * mhz * 1e6 / 1e12
    tflops = flops_per_lu * mlups * 1e6 / 1e12
    return {"oracle_flops_per_lu": flops_per_lu, "oracle_equivalent_tflops": tflops,
            "fp32_peak_tflops": peak, "frac": tflops / peak,
            "alu_bound_mlups_at_oracle_flops": peak * 1e12 / flops_per_lu / 1e6,
            "note": "peak derived from unit counts and the sampled max SM clock; the fused kernel "
                    "folds the arithmetic and executes fewer operations (FMA pipe use in profiles/)"}


def run(args):
    import torch

    import paper_2508_00577_gb300 as ev

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    layers = list(range(args.layers)) if args.layers < 9 else None
    (rho, u, T), nz = workload_fields(ev.lbm_coexistence, ev.lbm_critical_point, layers=layers)
    params = ev.lbm_params.make(lattice=ev.LBM_D2Q9, nx=NX, ny=NY, nz=nz, eos=ev.LBM_EOS_CS, a=A, b=B,
                                kappa=KAPPA, tau=TAU, lambda_=1.0, thermal=1, precision=ev.LBM_FP32)
    N = params.N
    lat = ev.Lattice(params, rho, u, T, stream=stream.cuda_stream)
    launches_per_step = ev.lbm_launches_per_step(lat.ctx)
    if args.tile:
        ev.lbm_set_tile(lat.ctx, *(int(v) for v in args.tile.split(",")))
        tile = ev.lbm_get_tile(lat.ctx)
    else:
        tile = ev.lbm_autotune(lat.ctx, 3) if not args.no_autotune else ev.lbm_get_tile(lat.ctx)

    # Warm-up
    lat.step(args.warmup)
    torch.cuda.synchronize(dev)
    c_start = lat.conserved()          # FP64 totals (outside the timed region)

    # Timed region: one event pair per step on the library's stream.
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            starts[k].record(stream)
            lat.step(1)
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    per_step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(sum(per_step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = job_mlups(world, N, args.steps, total_ms)

    c_end = lat.conserved()
    ok = np.isfinite(c_end).all()
    lat.close()
    conservation = {
        "mass_rel_drift": float(abs(c_end[0] - c_start[0]) / c_start[0]),
        "momentum_drift_per_node": float(np.abs(c_end[1:4] - c_start[1:4]).max() / N),
        "energy_population_rel_change": float((c_end[4] - c_start[4]) / c_start[4]),
        "over_steps": args.steps,
        "note": "FP64 totals of the FP32 state before and after the timed steps; the energy "
                "population changes by sum(u.F) per step (Eq. T_shift), mass and momentum are conserved"}

    # End to end through the public API with host buffers: init (H2D) + steps + moments (D2H).
    # The end-to-end job runs at least 2000 steps (a tenth of the sweep's 20000), so that a
    # short timed window (--steps) does not turn it into a measurement of lbm_init alone.
    e2e_steps = max(args.steps, 2000)
    pinned = [torch.from_numpy(a).pin_memory().numpy() for a in (rho, u.reshape(-1), T)]
    out_rho = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with ev.Lattice(params, pinned[0], pinned[1], pinned[2], stream=stream.cuda_stream) as lat2:
        ev.lbm_set_tile(lat2.ctx, *tile)
        lat2.step(e2e_steps)
        ev.lbm_moments(lat2.ctx, out_rho, None, None, None)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": N * e2e_steps / e2e_s / 1e6 * world, "unit": "MLUPS",
           "h2d_bytes_per_step": int(sum(a.nbytes for a in pinned) / e2e_steps),
           "d2h_bytes_per_step": int(out_rho.nbytes / e2e_steps),
           "what": f"lbm_init from host fields + {e2e_steps} x lbm_step + lbm_moments(rho) to host"}

    if rank != 0:
        return 0
    peak, peak_kind = peaks()
    achieved = BYTES_PER_LU * N / (ms_per_step * 1e-3) / 1e9
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if nz == 9 else f"{nz} of the 9 layers of: {WORKLOAD}", "nodes_per_gpu": N, "layers": nz, "lattice": "D2Q9",
                   "thermal": True, "precision": "fp32", "l2": "inputs larger than L2 (1.36 GB/step)",
                   "tile": {"w": tile[0], "h": tile[1], "autotuned": not (args.no_autotune or args.tile)},
                   "parallelism": f"replicas x{world}",
                   "quoted_on": "the 2-D static-droplet Laplace sweep (1024^2 periodic, FP32, T/Tc in {0.7, 0.8, "
                                "0.9} x R in {64, 128, 256}, one layer each), the workload the MLUPS headline is "
                                "quoted on; the 256^3 D3Q27 spinodal (FP32/FP16/BF16) and the 512-domain ensemble "
                                "follow as sub-lines of the same run"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (MEASURED_TRAFFIC_BYTES[tuple(tile)] / 1e9
                                 if nz == 9 and tuple(tile) in MEASURED_TRAFFIC_BYTES else None),
                     "traffic_unit": "GB per launch",
                     "note": f"{BYTES_PER_LU} algorithmic B/LU; peak {peak_kind} copy bandwidth"},
        "alu_check": alu_check(value, ORACLE_FLOPS_PER_LU["d2q9_thermal"], clk.summary().get("sm_max_mhz")),
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "finite": bool(ok),
        "conservation": conservation,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if world == 1 and not args.no_extra:
        # The other rows, measured on their own workloads: the batched persistent
        # ensemble (A11) and the 3-D path with reduced-precision storage (A10).
        eargs = argparse.Namespace(**vars(args))
        eargs.domains, eargs.steps, eargs.warmup, eargs.tile = 512, ENSEMBLE_STEPS, 20, ""
        e_line = run_ensemble(eargs)
        line["ensemble"] = {k: e_line[k] for k in ("metric", "value", "unit", "steps", "ms_per_step", "config",
                                                     "roofline", "finite", "finite_domains")}
        sargs3 = argparse.Namespace(**vars(args))
        sargs3.steps, sargs3.warmup, sargs3.tile = 20, 3, ""
        line["spinodal3d"] = run_spinodal3d(sargs3)
        line["sweep_fp16_bf16"] = run_sweep16(sargs3)
        # Physics checks of the same kernels (not timed): the Laplace law of droplets and
        # the paper's supersonic thermal Couette flow.
        line["laplace"] = {k: v for k, v in run_laplace(args).items() if k not in ("data",)}
        line["couette"] = {k: v for k, v in run_couette(args).items() if k not in ("data",)}
    if world == 1 and not args.no_surrogate:
        # The learned-surrogate row: speedup of surrogate + fallback over the plain
        # LB at <= 1e-2 relative density error (separate workload, see run_surrogate).
        sargs = argparse.Namespace(**vars(args))
        sargs.domains, sargs.warmup = 32, 20
        s_line = run_surrogate(sargs)
        line["surrogate"] = {k: s_line[k] for k in ("metric", "value", "unit", "meets_rho_rel_l2_1e-2", "config",
                                                      "plain_lb_seconds", "rollouts", "inference", "training")}
    emit(line, args)
    return 0


def run_sweep16(args):
    """The headline sweep (9 x 1024^2 D2Q9 thermal) with FP16 / BF16 deviation storage on
    the same fused kernel (120 algorithmic B/LU: 16-bit populations and the 24-byte
    reference records), timed like the headline: CUDA events on the library's stream."""
    import torch

    import paper_2508_00577_gb300 as ev

    (rho, u, T), nz = workload_fields(ev.lbm_coexistence, ev.lbm_critical_point)
    peak, peak_kind = peaks()
    out = {"config": {"workload": WORKLOAD.replace("FP32", "FP16/BF16 deviation storage"),
                      "peak": f"{peak:.1f} GB/s ({peak_kind})"}}
    for prec, name in ((ev.LBM_FP16_DEV, "fp16"), (ev.LBM_BF16_DEV, "bf16")):
        p = ev.lbm_params.make(lattice=ev.LBM_D2Q9, nx=NX, ny=NY, nz=nz, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=KAPPA,
                               tau=TAU, lambda_=1.0, thermal=1, precision=prec)
        stream = torch.cuda.Stream()
        with ev.Lattice(p, rho, u, T, stream=stream.cuda_stream) as g:
            if args.tile:                       # fixed W,H launch shape (the one a profile captures)
                ev.lbm_set_tile(g.ctx, *(int(v) for v in args.tile.split(",")))
                tile = ev.lbm_get_tile(g.ctx)
            else:
                tile = ev.lbm_autotune(g.ctx, 3)
            g.step(args.warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            g.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            finite = bool(np.isfinite(g.conserved()).all())
            launches = ev.lbm_launches_per_step(g.ctx)
        nodes = NX * NY * nz
        gbs = 120 * nodes / (ms * 1e-3) / 1e9
        out[name] = {"mlups": nodes / (ms * 1e-3) / 1e6, "ms_per_step": ms, "launches_per_step": launches,
                     "tile": list(tile), "algorithmic_bytes_per_lu": 120, "achieved_gbs": gbs, "frac": gbs / peak,
                     "finite": finite}
    return out


def run_ensemble(args):
    """512 independent 2-D droplet-pair domains of uneven sizes (64..512 per side), FP32
    thermal, all advanced by one persistent launch per call under a CUDA graph."""
    import torch

    import paper_2508_00577_gb300 as ev
    from paper_2508_00577_gb300 import inputs

    _, Tc = ev.lbm_critical_point(1, A, B)
    doms = inputs.ensemble_domains(args.domains)
    cache = {}
    rho, u, T, sizes = [], [], [], []
    for dm in doms:
        tr = round(dm["tr"], 3)
        if tr not in cache:
            cache[tr] = ev.lbm_coexistence(1, A, B, tr * Tc)
        rv, rl = cache[tr]
        r, v, t = inputs.two_droplets(dm["nx"], dm["ny"], dm["r1"], dm["r2"], dm["gap"], rv, rl, dm["tr"] * Tc)
        rho.append(r); u.append(v); T.append(t); sizes.append((dm["nx"], dm["ny"]))
    params = ev.lbm_params.make(eos=ev.LBM_EOS_CS, a=A, b=B, kappa=ENSEMBLE_KAPPA, tau=TAU, thermal=1,
                                precision=ev.LBM_FP32)
    stream = torch.cuda.Stream()
    bt = ev.Batch(params, sizes, rho, u, T, stream=stream.cuda_stream)
    if args.tile:                       # fixed W,H launch shape (the one a profile captures)
        tile = tuple(int(v) for v in args.tile.split(","))
        bt.set_tile(*tile)
    else:
        tile = bt.autotune(8)            # 16-step probe launches: a run is thousands of steps
    bt.step(args.warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0.record(stream)
        bt.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    N = bt.nodes()
    value = N * args.steps / (ms * 1e-3) / 1e6
    peak, peak_kind = peaks()
    achieved = BYTES_PER_LU * N * args.steps / (ms * 1e-3) / 1e9
    # Every domain is checked: a few coalescing pairs near T/Tc = 0.7 leave the method's
    # stability range within a few hundred steps (the FP64 oracle diverges on them too);
    # their NaN arithmetic costs the same on the GPU, and the count is reported.
    n_finite = sum(bool(np.isfinite(bt.moments(d)[0]).all()) for d in range(len(sizes)))
    bt.close()
    return {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"ensemble: {len(sizes)} uneven D2Q9 thermal domains (64..512)^2, FP32, "
                               f"kappa {ENSEMBLE_KAPPA}, {args.steps} steps in one persistent launch under a CUDA graph",
                   "nodes": N, "tile": {"w": tile[0], "h": tile[1], "autotuned": not args.tile}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": (ENSEMBLE_TRAFFIC_BYTES_PER_STEP[tuple(tile)] / 1e9
                                 if len(sizes) == 512 and tuple(tile) in ENSEMBLE_TRAFFIC_BYTES_PER_STEP else None),
                     "traffic_unit": "GB per step (ncu, one-step launch)",
                     "note": f"{BYTES_PER_LU} algorithmic B/LU; peak {peak_kind}"},
        "clocks": clk.summary(), "gpu_launches": 1, "finite": n_finite == len(sizes),
        "finite_domains": f"{n_finite}/{len(sizes)}",
    }


# Surrogate workload (A12): droplet-pair domains of 256^2 drawn like the ensemble's
# (radii U[8, 48], gap U[2, 10], T/Tc U[0.7, 0.9]); kappa = 0.2 (10-90 % width 5.3 at
# T/Tc = 0.7, 9.6 at 0.9) because at kappa = 0.116 about 5 % of these domains diverge
# before 5000 steps; windows of 50 steps.
SUR_N, SUR_KAPPA, SUR_STEPS, SUR_WINDOWS = 256, 0.2, 50, 100


def surrogate_fields(ev, doms, Tc):
    from paper_2508_00577_gb300 import inputs
    cache, rho, T = {}, [], []
    for dm in doms:
        tr = round(dm["tr"], 4)
        if tr not in cache:
            cache[tr] = ev.lbm_coexistence(1, A, B, tr * Tc)
        rv, rl = cache[tr]
        r, _, t = inputs.two_droplets(SUR_N, SUR_N, dm["r1"], dm["r2"], dm["gap"], rv, rl, dm["tr"] * Tc)
        rho.append(r)
        T.append(t)
    rho, T = np.concatenate(rho), np.concatenate(T)
    return rho, np.zeros((2, rho.size)), T


def run_surrogate(args):
    """Train the U-Net surrogate on lattice Boltzmann trajectories, then compare the
    time to solution of a 5000-step rollout (surrogate windows with lattice Boltzmann
    fallback) with the plain FP32 lattice Boltzmann run on held-out domains."""
    import torch

    import paper_2508_00577_gb300 as ev
    from paper_2508_00577_gb300 import inputs
    from paper_2508_00577_gb300 import surrogate as S

    dev = "cuda"
    _, Tc = ev.lbm_critical_point(1, A, B)
    Mb = SUR_N * SUR_N

    def params(nd):
        return ev.lbm_params.make(nx=SUR_N, ny=SUR_N, nz=nd, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=SUR_KAPPA, tau=TAU,
                                  precision=ev.LBM_FP32)

    def trajectories(doms):
        nd = len(doms)
        N = nd * Mb
        snaps = torch.empty((SUR_WINDOWS + 1, 4, N), device=dev)
        with ev.Lattice(params(nd), *surrogate_fields(ev, doms, Tc)) as g:
            for w in range(SUR_WINDOWS + 1):
                if w:
                    g.step(SUR_STEPS)
                base = snaps.data_ptr() + w * 16 * N
                ev.lbm_moments_device(g.ctx, base, base + 4 * N, base + 12 * N)
            ev.lbm_sync(g.ctx)
        torch.cuda.synchronize()
        return snaps

    train_doms = inputs.ensemble_domains(args.train_domains, seed=1, side_min=SUR_N, side_max=SUR_N)
    test_doms = inputs.ensemble_domains(args.domains, seed=2, side_min=SUR_N, side_max=SUR_N)
    t0 = time.perf_counter()
    snaps = trajectories(train_doms)
    t_data = time.perf_counter() - t0
    x, y = snaps[:-1], snaps[1:]
    mean = x.mean(dim=(0, 2)).cpu().numpy()
    scale = np.maximum(x.std(dim=(0, 2)).cpu().numpy(), 1e-6)
    oscale = np.maximum((y - x).std(dim=(0, 2)).cpu().numpy(), 1e-9)
    view = snaps.reshape(SUR_WINDOWS + 1, 4, len(train_doms), Mb)
    bs = args.batch

    def batch(v, w, d):
        w = torch.as_tensor(w, device=dev)
        d = torch.as_tensor(d, device=dev)
        xb = v[w, :, d, :].permute(1, 0, 2).reshape(4, -1).contiguous()
        yb = v[w + 1, :, d, :].permute(1, 0, 2).reshape(4, -1).contiguous()
        return xb, yb

    def sequence(v, w, d, k):
        """Start fields of windows w and the k following states, [k][4][bs*Mb] targets."""
        w = torch.as_tensor(w, device=dev)
        d = torch.as_tensor(d, device=dev)
        x0 = v[w, :, d, :].permute(1, 0, 2).reshape(4, -1).contiguous()
        tg = torch.stack([v[w + j, :, d, :].permute(1, 0, 2).reshape(4, -1) for j in range(1, k + 1)]).contiguous()
        return x0, tg

    # A fixed validation batch from the first held-out domains, windows spread over the run.
    val = trajectories(test_doms[:8]).reshape(SUR_WINDOWS + 1, 4, 8, Mb)
    vx, vy = batch(val, np.arange(0, SUR_WINDOWS, SUR_WINDOWS // bs)[:bs], np.arange(bs) % 8)
    K = max(1, args.unroll)
    vsx, vst = sequence(val, np.arange(0, SUR_WINDOWS - K, (SUR_WINDOWS - K) // bs)[:bs], np.arange(bs) % 8, K)
    del val
    rng = np.random.default_rng(0)
    model = S.Surrogate(SUR_N, SUR_N, seed=3)
    model.set_norm(mean, scale, oscale)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for it in range(args.train_steps):
        xb, yb = batch(view, rng.integers(0, SUR_WINDOWS, bs), rng.integers(0, len(train_doms), bs))
        torch.cuda.synchronize()
        warm = min(1.0, (it + 1) / 200.0)
        lr = args.lr * warm * 0.5 * (1 + np.cos(np.pi * it / args.train_steps))
        want = it % 500 == 0 or it == args.train_steps - 1
        loss = model.train_step(xb.data_ptr(), yb.data_ptr(), bs, float(lr), want_loss=want)
        if want:
            losses.append((it, round(loss, 5), round(model.forward_backward(vx.data_ptr(), vy.data_ptr(), bs), 5)))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    # Unrolled fine-tuning: K windows applied to the network's own predictions, so that the
    # training sees (and is penalised for) the error it accumulates over a rollout.
    def val_losses():
        return (round(model.forward_backward(vx.data_ptr(), vy.data_ptr(), bs), 5),
                round(model.forward_backward_unrolled(vsx.data_ptr(), vst.data_ptr(), K, bs), 5))
    unrolled = {"windows": K, "steps": args.unroll_steps, "val_before": val_losses()}
    t0 = time.perf_counter()
    for it in range(args.unroll_steps):
        x0, tg = sequence(view, rng.integers(0, SUR_WINDOWS - K + 1, bs), rng.integers(0, len(train_doms), bs), K)
        torch.cuda.synchronize()
        lr = 0.3 * args.lr * 0.5 * (1 + np.cos(np.pi * it / args.unroll_steps))
        model.train_step_unrolled(x0.data_ptr(), tg.data_ptr(), K, bs, float(lr), want_loss=False)
    torch.cuda.synchronize()
    unrolled["seconds"] = time.perf_counter() - t0
    unrolled["val_after"] = val_losses()
    unrolled["val_note"] = f"(one-window loss, {K}-window unrolled loss) on held-out windows"
    del snaps, view, x, y, vx, vy, vsx, vst

    # Held-out domains: the plain lattice Boltzmann run is the reference every error is measured against.
    nd = len(test_doms)
    N = nd * Mb
    rho0, u0, T0 = surrogate_fields(ev, test_doms, Tc)
    steps = SUR_STEPS * SUR_WINDOWS
    ref = torch.empty((4, N), device=dev)
    with ev.Lattice(params(nd), rho0, u0, T0) as g:
        tile = ev.lbm_autotune(g.ctx, 2)
        g.step(args.warmup)
        torch.cuda.synchronize()
    with ev.Lattice(params(nd), rho0, u0, T0) as g:
        ev.lbm_set_tile(g.ctx, *tile)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(steps)
        ev.lbm_moments_device(g.ctx, ref.data_ptr(), ref.data_ptr() + 4 * N, ref.data_ptr() + 12 * N)
        ev.lbm_sync(g.ctx)
        torch.cuda.synchronize()
        t_lb = time.perf_counter() - t0
    start = torch.tensor(np.stack([rho0, u0[0], u0[1], T0]), dtype=torch.float32, device=dev).contiguous()
    rho_mid = float(0.5 * (start[0].max() + start[0].min()))

    def rel_err(a):
        per = [float((a[0, k * Mb:(k + 1) * Mb] - ref[0, k * Mb:(k + 1) * Mb]).norm()
                     / ref[0, k * Mb:(k + 1) * Mb].norm()) for k in range(nd)]
        return float((a[0] - ref[0]).norm() / ref[0].norm()), max(per)

    # Rollouts: the surrogate alone, and with the fallback at a sweep of liquid-count
    # thresholds (mass projected, so the mass indicator is a safeguard only).
    configs = [("surrogate_only", 1e30, 1e30, False, 1.0)]
    configs += [(f"fallback_area_{a:g}", args.max_mass_drift, a, True, 1.0) for a in args.area_sweep]
    configs += [(f"fallback_interface_{f:g}", args.max_mass_drift, 1e30, True, f) for f in args.shift_sweep]
    results = {}
    for name, dm, da, proj, shift in configs:
        with ev.Lattice(params(nd), rho0, u0, T0) as lb:
            ev.lbm_set_tile(lb.ctx, *tile)
            d = start.clone()
            model.infer(d.data_ptr(), torch.empty_like(d).data_ptr(), nd)   # warm the arena
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                nfb, used = model.rollout(lb.ctx, d.data_ptr(), nd, SUR_WINDOWS, SUR_STEPS, rho_mid, dm, da, proj, shift)
                failed = None
            except S.SurError as exc:
                nfb, failed = -1, str(exc)
            torch.cuda.synchronize()
            t_roll = time.perf_counter() - t0
        err, worst = rel_err(d)
        results[name] = {"seconds": t_roll, "speedup_vs_lb": t_lb / t_roll, "fallback_windows": int(nfb),
                         "rho_rel_l2": err, "rho_rel_l2_worst_domain": worst, "failed": failed}
    ok = [r for r in results.values() if r["failed"] is None and r["rho_rel_l2"] <= 1e-2]
    best = max(ok, key=lambda r: r["speedup_vs_lb"]) if ok else None
    # Inference throughput alone.
    o = torch.empty_like(start)
    for _ in range(3):
        model.infer(start.data_ptr(), o.data_ptr(), nd)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        model.infer(start.data_ptr(), o.data_ptr(), nd)
    torch.cuda.synchronize()
    t_inf = (time.perf_counter() - t0) / 10
    flops = 17.93e9 * nd
    model.close()
    line = {
        "metric": "surrogate+fallback time-to-solution speedup vs plain FP32 LB at rho rel. L2 <= 1e-2",
        "value": best["speedup_vs_lb"] if best else None,
        "unit": "x", "n_gpus": 1, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
        "meets_rho_rel_l2_1e-2": best is not None,
        "config": {"workload": f"{nd} held-out droplet-pair domains of {SUR_N}^2, {steps} steps = {SUR_WINDOWS} windows "
                               f"of {SUR_STEPS}; trained on {len(train_doms)} domains x {SUR_WINDOWS} windows",
                   "kappa": SUR_KAPPA, "tau": TAU, "train_steps": args.train_steps, "batch": bs,
                   "max_mass_drift": args.max_mass_drift, "area_sweep": args.area_sweep,
                   "interface_shift_sweep": args.shift_sweep},
        "plain_lb_seconds": t_lb, "plain_lb_mlups": N * steps / t_lb / 1e6,
        "rollouts": results,
        "inference": {"ms_per_window": t_inf * 1e3, "tflops": flops / t_inf / 1e12, "batch": nd},
        "training": {"seconds": t_train, "ms_per_step": t_train / args.train_steps * 1e3, "data_seconds": t_data,
                     "unrolled": unrolled,
                     "loss_train_val": losses},
    }
    return line


def run_spinodal3d(args):
    """3-D spinodal decomposition, 256^3 D3Q27 thermal: mean density at the midpoint of
    the spinodal region at T/Tc = 0.85 with seeded uniform +-1 % noise, u = 0; FP32
    storage and arithmetic, and FP16 / BF16 deviation storage with FP32 arithmetic.
    One line with MLUPS and the fraction of the HBM roofline per storage type
    (algorithmic bytes: 2 populations x 27 x read + write x storage bytes, plus for
    16-bit storage the 24-byte FP32 reference record of every node, read and written)."""
    import torch

    import paper_2508_00577_gb300 as ev
    from paper_2508_00577_gb300 import inputs

    n = args.n3d
    _, Tc = ev.lbm_critical_point(ev.LBM_EOS_CS, A, B)
    RT = 0.85 * Tc
    s1, s2 = ev.lbm_spinodal(ev.LBM_EOS_CS, A, B, RT)
    kappa = ev.lbm_kappa_for_width(ev.LBM_EOS_CS, A, B, RT, 4.0)
    rho, u, T = inputs.spinodal_noise(n, n, n, 0.5 * (s1 + s2), RT, amplitude=0.01)
    peak, peak_kind = peaks()
    out = {}
    for prec, name, sb in ((ev.LBM_FP32, "fp32", 4), (ev.LBM_FP16_DEV, "fp16", 2), (ev.LBM_BF16_DEV, "bf16", 2)):
        p = ev.lbm_params.make(lattice=ev.LBM_D3Q27, nx=n, ny=n, nz=n, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa,
                               tau=TAU, precision=prec)
        stream = torch.cuda.Stream()
        with ev.Lattice(p, rho, u, T, stream=stream.cuda_stream) as g:
            if args.tile:                            # fixed z-chunk H (--tile W,H: W is the kernel's own)
                ev.lbm_set_tile(g.ctx, 0, int(args.tile.split(",")[-1]))
                tile = ev.lbm_get_tile(g.ctx)
            else:
                tile = ev.lbm_autotune(g.ctx, 2)     # z-chunk of the fused kernel
            g.step(args.warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            g.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            launches = ev.lbm_launches_per_step(g.ctx)
            finite = bool(np.isfinite(g.conserved()).all())
        bpl = 2 * 27 * 2 * sb + (2 * 24 if sb == 2 else 0)
        out[name] = {"mlups": p.N / (ms * 1e-3) / 1e6, "ms_per_step": ms, "launches_per_step": launches,
                     "tile": tile,
                     "algorithmic_bytes_per_lu": bpl, "achieved_gbs": bpl * p.N / (ms * 1e-3) / 1e9,
                     "frac": bpl * p.N / (ms * 1e-3) / 1e9 / peak, "finite": finite}
        if prec == ev.LBM_FP32:
            out[name]["alu_check"] = alu_check(out[name]["mlups"], ORACLE_FLOPS_PER_LU["d3q27_thermal"])
    return {"metric": "MLUPS", "value": out["fp32"]["mlups"], "unit": "MLUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"3-D spinodal decomposition, {n}^3 D3Q27 thermal, T/Tc = 0.85",
                       "peak": f"{peak} GB/s ({peak_kind})"},
            "by_storage": out}


def run_coexistence(args):
    """The paper's Fig. 1 setting on the fused FP32 kernel: isothermal van der Waals slabs
    (a = 9/392/16, b = 2/21, 8-node interfaces, 8000 steps) over T/Tc = 0.6..0.95; the
    coexistence densities next to the Maxwell construction of the same EOS."""
    import paper_2508_00577_gb300 as ev
    from paper_2508_00577_gb300 import inputs

    a, b = 9 / 392 / 16, 2 / 21
    _, Tc = ev.lbm_critical_point(ev.LBM_EOS_VDW, a, b)
    curve = []
    for tr in (0.6, 0.65, 0.7, 0.75, 0.8, 0.85, 0.9, 0.95):
        RT = tr * Tc
        rv, rl = ev.lbm_coexistence(ev.LBM_EOS_VDW, a, b, RT)
        kappa = ev.lbm_kappa_for_width(ev.LBM_EOS_VDW, a, b, RT, 8.0)
        f = inputs.slab(384, 4, rv, rl, RT, thickness=192.0, width=8.0)
        p = ev.lbm_params.make(nx=384, ny=4, eos=ev.LBM_EOS_VDW, a=a, b=b, kappa=kappa, tau=TAU, thermal=0,
                               precision=ev.LBM_FP32)
        with ev.Lattice(p, *f) as g:
            g.step(8000)
            rho = g.moments()[0]
        fin = bool(np.isfinite(rho).all())
        curve.append({"T_over_Tc": tr, "rho_liquid": float(rho.max()) if fin else None, "rho_vapour":
                      float(rho.min()) if fin else None, "maxwell_liquid": rl, "maxwell_vapour": rv, "finite": fin})
    return {"metric": "coexistence curve (Fig. 1 setting)", "unit": "lattice density", "data": "synthetic",
            "config": {"workload": "isothermal vdW slabs 384 x 4, a = 9/392/16, b = 2/21, width 8, 8000 steps, "
                                   "fused FP32 D2Q9 kernel"}, "curve": curve}


def cs_pressure(RT, rho, a=A, b=B):
    """p = P_E - a rho^2 of the Carnahan-Starling fluid (eta = b rho / 4)."""
    eta = b * np.asarray(rho) / 4.0
    return rho * RT * (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3 - a * np.asarray(rho) ** 2


def run_laplace(args):
    """Laplace law on the fused FP32 D2Q9 kernel: isothermal Carnahan-Starling droplets at
    T/Tc = 0.9 with 12-node interfaces (bare tau = 3), radii 36 and 48 in boxes of 2R + 40,
    6000 steps, pressure jump time-averaged over the second half; the slope of the jump
    against 1/R (through the origin, equimolar radius) next to the tension of a relaxed flat
    slab on the same kernel and to the square-gradient sigma of the library's interface
    solution (lbm_interface)."""
    import paper_2508_00577_gb300 as ev
    from paper_2508_00577_gb300 import inputs

    width, tau, tr = 12.0, 3.0, 0.9
    _, Tc = ev.lbm_critical_point(ev.LBM_EOS_CS, A, B)
    RT = tr * Tc
    rv, rl = ev.lbm_coexistence(ev.LBM_EOS_CS, A, B, RT)
    kappa = ev.lbm_kappa_for_width(ev.LBM_EOS_CS, A, B, RT, width)
    sigma = ev.lbm_interface(ev.LBM_EOS_CS, A, B, RT, kappa)[1]
    n = int(12 * width) + 48
    f = inputs.slab(n, 1, rv, rl, RT, thickness=n / 2, width=width)
    ps = ev.lbm_params.make(nx=n, ny=1, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa, tau=tau, thermal=0,
                            precision=ev.LBM_FP32)
    with ev.Lattice(ps, *f) as g:
        g.step(16000)
        rs = g.moments()[0]
    d = 0.5 * (np.roll(rs, -1) - np.roll(rs, 1))
    sig_m = 0.5 * kappa * float(np.sum(d * d))
    jumps = []
    for R in (36, 48):
        m = 2 * R + 40
        f = inputs.droplet(m, m, float(R), rv, rl, RT, width=width)
        pd = ev.lbm_params.make(nx=m, ny=m, eos=ev.LBM_EOS_CS, a=A, b=B, kappa=kappa, tau=tau, thermal=0,
                                precision=ev.LBM_FP32)
        acc = []
        with ev.Lattice(pd, *f) as g:
            for k in range(600):
                g.step(10)
                if k >= 300:
                    r = g.moments()[0].reshape(m, m)
                    c = m // 2
                    rin, rout = r[c - 2:c + 2, c - 2:c + 2].mean(), r[0:2, :].mean()
                    Re = np.sqrt((r.sum() - rout * m * m) / (rin - rout) / np.pi)
                    acc.append((cs_pressure(RT, rin) - cs_pressure(RT, rout), Re))
        dp, Re = np.mean(np.array(acc), axis=0)
        jumps.append({"R": R, "R_equimolar": float(Re), "dp": float(dp), "dp_R_over_sigma_model": float(dp * Re / sig_m),
                      "dp_R_over_sigma": float(dp * Re / sigma)})
    dps = np.array([j["dp"] for j in jumps])
    Res = np.array([j["R_equimolar"] for j in jumps])
    slope = float(np.sum(dps / Res) / np.sum(1.0 / Res**2))
    return {"metric": "Laplace law: slope of the pressure jump against 1/R", "value": slope, "unit": "lattice",
            "data": "synthetic", "slope_over_sigma_model": slope / sig_m, "slope_over_sigma": slope / sigma,
            "sigma_model": sig_m, "sigma": sigma, "jumps": jumps,
            "config": {"workload": "isothermal CS droplets R = 36, 48, T/Tc 0.9, 12-node interfaces, tau 3, "
                                   "6000 steps, fused FP32 D2Q9 kernel"}}


def run_couette(args):
    """The paper's supersonic thermal Couette flow (Fig. 2 set-up) on the fused FP32 D2Q9
    kernel with diffusely reflecting wall nodes (lbm_set_walls): a van der Waals gas
    (b = 0.1, a = 0.05, rho = 1, R T_w = 0.2), Ma = 1.2 at the moving wall, channel of 65
    nodes, bare tau = 0.5, 100000 steps; the steady profile next to T(u_y) = T_w +
    u_y (U_w - u_y) / 5 (the Navier-Stokes-Fourier solution with k = 5/2 R mu)."""
    import paper_2508_00577_gb300 as ev

    b, a, RTw, Ma, nx, tau = 0.1, 0.05, 0.2, 1.2, 66, 0.5
    Z = 1.0 / (1.0 - b)
    g0 = 5.0 / 3.0 * Z
    Uw = Ma * float(np.sqrt(g0 * RTw * Z - 2 * a))        # adiabatic sound speed of p = P_E - a rho^2 at rho = 1
    u = np.zeros((2, nx))
    u[1, -1] = Uw
    p = ev.lbm_params.make(nx=nx, ny=1, eos=ev.LBM_EOS_VDW, a=a, b=b, kappa=0.0, tau=tau, thermal=1,
                           precision=ev.LBM_FP32)
    with ev.Lattice(p, np.ones(nx), u, np.full(nx, RTw)) as g:
        ev.lbm_set_walls(g.ctx, 1, (0, 0, 0), (0, Uw, 0), RTw)
        g.step(100000)
        rho, uu, T, _ = g.moments()
    uy = uu[1]
    fl = slice(1, nx - 1)
    heat = Uw**2 / 20.0
    Tu = RTw + uy * (Uw - uy) / 5.0
    pr = rho * T / (1 - b * rho) - a * rho**2
    cs = np.sqrt(5.0 / 3.0 / (1 - b * rho[-2]) * T[-2] / (1 - b * rho[-2]) - 2 * a * rho[-2])
    return {"metric": "thermal Couette flow: max |T - T(u_y)| / viscous heating", "value":
            float(np.abs(T - Tu)[fl].max() / heat), "unit": "fraction", "data": "synthetic",
            "mach_at_moving_wall": float(uy[-2] / cs), "U_w": Uw,
            "pressure_spread": float((pr[fl].max() - pr[fl].min()) / pr[fl].mean()),
            "T_mid_minus_Tw_over_heating": float((T[nx // 2] - RTw) / heat),
            "config": {"workload": "vdW gas b 0.1, a 0.05, 65-node channel, Ma 1.2, tau 0.5, 100000 steps, "
                                   "fused FP32 D2Q9 kernel with wall nodes"}}


def run_surrogate_kernels(args):
    """Kernel-level timing of the surrogate on batch --batch of 256^2 domains: two
    inferences and one training step (the case the ncu summaries capture), then
    CUDA-event timing of each over --steps repetitions."""
    import torch

    from paper_2508_00577_gb300 import surrogate as S

    dev = "cuda"
    bs, n = args.batch, SUR_N
    r = np.random.default_rng(0)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    base = np.stack([np.sin(2 * np.pi * (k + 1) * yy / n + k) * np.cos(2 * np.pi * xx / n) for k in range(4)])
    x = np.concatenate([base.reshape(4, -1)] * bs, axis=1) * np.array([[0.05], [0.004], [0.004], [0.0005]])
    x += np.array([[0.1], [0.0], [0.0], [0.0075]]) + 1e-4 * r.standard_normal(x.shape)
    dx = torch.tensor(x, dtype=torch.float32, device=dev).contiguous()
    dy = dx + 1e-4
    out = torch.empty_like(dx)
    m = S.Surrogate(n, n, seed=3)
    m.set_norm([0.1, 0, 0, 0.0075], [0.05, 0.004, 0.004, 0.0005], [0.002, 0.001, 0.001, 8e-5])
    torch.cuda.synchronize()
    for _ in range(2):
        m.infer(dx.data_ptr(), out.data_ptr(), bs)
    m.train_step(dx.data_ptr(), dy.data_ptr(), bs, 1e-4, want_loss=False)
    torch.cuda.synchronize()
    res = {}
    for name, fn in (("infer", lambda: m.infer(dx.data_ptr(), out.data_ptr(), bs)),
                     ("train_step", lambda: m.train_step(dx.data_ptr(), dy.data_ptr(), bs, 1e-4, want_loss=False))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fn()
        torch.cuda.synchronize()
        res[name] = (time.perf_counter() - t0) / args.steps * 1e3
    m.close()
    flops = 17.93e9 * bs
    emit({"metric": "surrogate inference TFLOP/s", "value": flops / res["infer"] / 1e9, "unit": "TFLOP/s",
                      "n_gpus": 1, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
                      "config": {"workload": f"U-Net on {bs} x {n}^2 domains", "batch": bs},
                      "ms_per_inference": res["infer"], "ms_per_train_step": res["train_step"],
                      "train_tflops": 3 * flops / res["train_step"] / 1e9,
                      "bf16_peak_tflops": peaks_bf16()}, args)
    return 0


def peaks_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 2000; ensemble: its full 5000)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--layers", type=int, default=9, help="layers of the sweep (9 = the full workload)")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate measurement in the default run")
    ap.add_argument("--no-extra", action="store_true", help="skip the ensemble and 3-D measurements in the default run")
    ap.add_argument("--tile", default="", help="fixed launch shape W,H of the fused kernel")
    ap.add_argument("--log", default="", help="also append each result line to this JSON-lines file")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "sweep16", "ensemble", "surrogate", "surrogate_kernels",
                                                         "spinodal3d", "laplace", "couette",
                                                           "coexistence"],
                    help="sweep: the headline droplet Laplace sweep; ensemble: 512 uneven domains; "
                         "surrogate: U-Net surrogate with lattice Boltzmann fallback vs plain LB")
    ap.add_argument("--n3d", type=int, default=256, help="spinodal3d: cube side")
    ap.add_argument("--domains", type=int, default=None, help="ensemble: 512; surrogate: 32 held-out domains")
    ap.add_argument("--train-domains", type=int, default=64)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--unroll", type=int, default=4, help="surrogate: windows of the unrolled fine-tuning")
    ap.add_argument("--unroll-steps", type=int, default=1000, help="surrogate: unrolled fine-tuning steps (0: none)")
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--max-mass-drift", type=float, default=1e-3)
    ap.add_argument("--area-sweep", type=float, nargs="+", default=[0.02, 0.005, 0.001])
    ap.add_argument("--shift-sweep", type=float, nargs="+", default=[0.01, 0.002],
                    help="surrogate: thresholds of the interface-position indicator (fraction of nodes changing phase)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = ENSEMBLE_STEPS if args.workload == "ensemble" and args.impl == "native" else 2000
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        args.domains = args.domains or 512
        emit(run_ensemble(args), args)
        return 0
    if args.workload == "surrogate":
        args.domains = args.domains or 32
        emit(run_surrogate(args), args)
        return 0
    if args.workload == "surrogate_kernels":
        return run_surrogate_kernels(args)
    if args.workload == "spinodal3d":
        emit(run_spinodal3d(args), args)
        return 0
    if args.workload == "sweep16":
        line = run_sweep16(args)
        line.update({"metric": "MLUPS", "value": line["fp16"]["mlups"], "unit": "MLUPS", "n_gpus": 1,
                     "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f16",
                     "data": "synthetic"})
        emit(line, args)
        return 0
    if args.workload == "coexistence":
        emit(run_coexistence(args), args)
        return 0
    if args.workload == "laplace":
        emit(run_laplace(args), args)
        return 0
    if args.workload == "couette":
        emit(run_couette(args), args)
        return 0
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
