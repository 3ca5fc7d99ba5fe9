"""Benchmark of the NDG + RK hot path on B300: DOF-updates per second per RK stage.

Workload (one bench step): the 2D linear advection problem of the paper's Sec. 3 at degree 7,
256 x 256 quadrilateral elements (8 x 8 LGL nodes each, 2048^2 = 4.19M DOF), velocity (1, 0.5),
Gaussian pulse exp(-r^2/0.01) at the centre plus seeded low-mode Fourier noise (amplitude 1e-3),
upwind flux, classical RK4 at CFL 0.1, 1000 time steps, followed by the norms reduction.  The
state is reset from a device-resident copy of the initial condition and L2 is flushed at the start
of every bench step.  FP64 is the headline; the FP32 variant and a mixed serving stream are
reported beside it; the FP64 CPU oracle (single thread, as it stands) gives the CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-serving]
                    [--no-workloads] [--workload adv2d|euler2d|euler3d|euler3d7] [--variants f64,f32,f64ff]

Beside the headline, the line carries a table of the isothermal Euler problems (2D 512^2 at
degree 7, 3D 64^3 at degree 5, 3D 32^3 at degree 7): FP64 and FP32 ms per stage with their
roofline fractions.

Under torchrun (N > 1) every rank runs an independent replica of the workload ("replicas only":
the solve is not partitioned across GPUs); value = total DOF-updates / max rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RK stage (FP64 vs FP32); batched solves/s + p50/p99 latency"
# The bench workload (default) and the other full-size problems, selectable with
# --workload: (dim, degree, elements, equation, velocity, RK steps per bench step, description).
WORKLOADS = {
    "adv2d": (2, 7, (256, 256), 0, (1.0, 0.5, 0.0), 1000,
              "2D linear advection, 256x256 elements, degree 7 (8x8 LGL nodes), 4.19M DOF, RK4, 1000 steps"),
    "euler2d": (2, 7, (512, 512), 1, (0.0, 0.0, 0.0), 200,
                "2D isothermal Euler, 512x512 elements, degree 7, 3 x 4096^2 = 50.3M DOF, RK4, 200 steps"),
    "euler3d": (3, 5, (64, 64, 64), 1, (0.0, 0.0, 0.0), 50,
                "3D isothermal Euler, 64^3 elements, degree 5, 4 x 384^3 = 226.5M DOF, RK4, 50 steps"),
    # the eighth-order 3D case (degree 7) at the same size class
    "euler3d7": (3, 7, (32, 32, 32), 1, (0.0, 0.0, 0.0), 50,
                 "3D isothermal Euler, 32^3 elements, degree 7 (8^3 LGL nodes), 4 x 256^3 = 67.1M DOF, RK4, 50 steps"),
}
DIM, DEGREE, ELEMS, EQ, VEL, NSTEPS, WORKLOAD = WORKLOADS["adv2d"]
CFL, RK = 0.1, 4
STAGES = 4
L2_FLUSH_BYTES = 256 << 20


def select_workload(name):
    global DIM, DEGREE, ELEMS, EQ, VEL, NSTEPS, WORKLOAD
    DIM, DEGREE, ELEMS, EQ, VEL, NSTEPS, WORKLOAD = WORKLOADS[name]

# Algorithmic work of one RK4 stage per DOF:
#   flops, 2D advection degree 7: sum-factorised strong-form volume term 2 axes x 8 FMA (32 flop)
#          + per-axis scaling (3) + lifted face terms (1.5) + stage update (3.5 on average over the
#          4 stages) = 40 flop; 2D isothermal Euler degree 7: 48; 3D isothermal Euler degree 5: 60;
#          3D isothermal Euler degree 7: 72 (volume 3 axes x 8 FMA = 48 instead of 3 x 6 = 36);
#   bytes: RK4 array passes per stage 3, 5, 5, 3 -> 4 on average x sizeof(real).
FLOPS_PER_DOF = {"adv2d": 40.0, "euler2d": 48.0, "euler3d": 60.0, "euler3d7": 72.0}
# DRAM bytes per stage launch of the bench workload's kernels (mean of the four RK4 stages), from
# one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum (command and per-stage values in
# profiles/stage_kernel_2d_advection_deg7_256x256.md); to be captured again when the kernel changes.
TRAFFIC_PER_LAUNCH = {("adv2d", "f64"): 91.95e6, ("adv2d", "f32"): 37.79e6}
FLOPS_PER_DOF_STAGE = FLOPS_PER_DOF["adv2d"]
PASSES_PER_STAGE = 4.0


_T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    sys.stderr.write(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}\n")
    sys.stderr.flush()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def fp64_peak_tflops(sm_mhz):
    # 148 SMs x 2 DFMA / clock / SM x 2 flop (B300 FP64 units; 1.12 TFLOP/s measured at 1935 MHz)
    return 148 * 2 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
                self.lines = [l for l in out.splitlines() if l.strip()]
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons, power = [], 0.0, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except (ValueError, IndexError):
                continue
            try:
                power.append(float(f[3]))
            except (ValueError, IndexError):
                pass
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "power_w": statistics.median(power) if power else None}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg, dev=None):
    if pg is not None:
        if dev is not None:
            pg.barrier(device_ids=[dev])
        else:
            pg.barrier()


def max_over_ranks(pg, x, dev):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=f"cuda:{dev}" if dev is not None else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def data_description():
    """What the synthetic initial state of the selected workload is."""
    if EQ == 0:
        return "synthetic (seeded Gaussian pulse + Fourier noise)"
    if DIM == 2:
        return "synthetic (isothermal Euler: density 1 + 0.1 sin sin, seeded smooth shear velocity, Mach <= 0.3)"
    return "synthetic (isothermal Euler: density 1, Taylor-Green velocity of amplitude 0.1)"


def initial_condition(X):
    from paper_2510_05254_b300 import inputs
    if EQ == 0:
        return inputs.gaussian_noise(X)
    return inputs.euler_shear(X) if DIM == 2 else inputs.taylor_green(X)


def oracle_sample(nsteps):
    """The FP64 oracle as it stands (single thread) on the full workload for nsteps RK4 steps."""
    from oracle import oracle as orc
    p = orc.Problem(dim=DIM, degree=DEGREE, elems=tuple(ELEMS) + (1,) * (3 - DIM), equation=EQ, flux=EQ,
                    velocity=VEL)
    U0 = initial_condition(orc.node_coords(p))
    dt = orc.stable_dt(p, U0, CFL)
    t = time.perf_counter()
    orc.step(p, U0, dt, nsteps, RK)
    el = time.perf_counter() - t
    return p.ndof * STAGES * nsteps / el, el


def run_reference(args, world, rank):
    if rank != 0:
        return None
    sample_steps = 1
    for _ in range(args.warmup):
        oracle_sample(sample_steps)
    rates, tot = [], 0.0
    for _ in range(args.steps):
        r, el = oracle_sample(sample_steps)
        rates.append(r)
        tot += el
    value = statistics.median(rates)
    ndof = config_block(world)["dof"]
    sample = f"{sample_steps} RK4 step of the full {ndof / 1e6:.2f}M-DOF workload per bench step ({NSTEPS} in the GPU step)"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": data_description(), "config": config_block(world),
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def config_block(world):
    ndof = (1 if EQ == 0 else DIM + 1) * int(np.prod(ELEMS)) * (DEGREE + 1) ** DIM
    return {"workload": WORKLOAD, "model": f"NDG+RK4, dim {DIM}, degree {DEGREE}", "global_batch": world,
            "seq_len": None, "elements": list(ELEMS), "degree": DEGREE, "dof": ndof,
            "rk_steps_per_bench_step": NSTEPS, "parallelism": f"replicas{world}",
            "l2": f"flushed at the start of every bench step ({L2_FLUSH_BYTES >> 20} MiB write, inside the timed region)"}


def run_solver_timed(dtype, args, dev, pg, U0_host):
    """Device-timed bench steps of one dtype: returns per-step device ms and stage-kernel ms."""
    import torch
    from paper_2510_05254_b300.solver import Solver
    s = Solver(DIM, DEGREE, ELEMS, equation=EQ, velocity=VEL, dtype=dtype, device=dev)
    U0 = torch.tensor(U0_host, device=f"cuda:{dev}", dtype=s.torch_dtype)
    s.set_state(U0)
    dt = s.stable_dt(CFL)
    if args.epb:  # a fixed tile (profiler captures of the tuned configuration)
        s.close()
        s = Solver(DIM, DEGREE, ELEMS, equation=EQ, velocity=VEL, dtype=dtype, device=dev, elems_per_block=args.epb)
        s.set_state(U0)
        epb = args.epb
    else:
        epb, _ = s.autotune(RK)  # the library's tile autotuner (state is restored bitwise)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    from paper_2510_05254_b300 import native as nat

    def one(evs=None):
        with torch.cuda.stream(s.stream):
            flush.zero_()
        nat.ndg_set_state(s.ctx, U0.data_ptr(), s.state_bytes, True)
        if evs:
            evs[0].record(s.stream)
        nat.ndg_step(s.ctx, dt, NSTEPS, RK)
        if evs:
            evs[1].record(s.stream)
        return nat.ndg_norms(s.ctx)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize(dev)
    barrier(pg, dev)
    torch.cuda.synchronize(dev)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    inner = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(dev) as clk:
        start.record(s.stream)
        for k in range(args.steps):
            nr = one(inner[k])
        end.record(s.stream)
        torch.cuda.synchronize(dev)
    barrier(pg, dev)
    total_ms = start.elapsed_time(end)
    stage_ms = sum(a.elapsed_time(b) for a, b in inner) / (args.steps * NSTEPS * STAGES)
    out = {"total_ms": total_ms, "stage_ms": stage_ms, "ndof": s.ndof, "dt": dt, "clocks": clk.summary(), "epb": epb,
           "kernel": "line" if s.kernel == 1 else "line_var",
           "l2_norm": nr.l2, "mass": nr.integral[0], "state_bytes": s.state_bytes,
           "final": s.get_state()}  # after NSTEPS steps from U0 (accuracy of the precisions)
    s.close()
    return out


def run_e2e(args, dev, U0_host):
    """Same workload through the C ABI with HOST buffers: pinned H2D of the initial state, 1000 RK
    steps, D2H of the final state and of the norms, every bench step."""
    import torch
    from paper_2510_05254_b300 import native as nat
    from paper_2510_05254_b300.solver import Solver
    s = Solver(DIM, DEGREE, ELEMS, equation=EQ, velocity=VEL, dtype="f64", device=dev)
    src = torch.tensor(U0_host, dtype=torch.float64).pin_memory()
    dst = torch.empty_like(src).pin_memory()
    s.set_state(U0_host)
    dt = s.stable_dt(CFL)

    def one():
        nat.ndg_set_state(s.ctx, src.data_ptr(), s.state_bytes, False)
        nat.ndg_step(s.ctx, dt, NSTEPS, RK)
        nat.ndg_get_state(s.ctx, dst.data_ptr(), s.state_bytes, False)
        return nat.ndg_norms(s.ctx)

    for _ in range(max(1, args.warmup)):
        one()
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    for _ in range(args.steps):
        one()
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t
    nb = s.state_bytes
    s.close()
    return el, nb


def run_serving(args, dev):
    from paper_2510_05254_b300 import inputs, serving
    n = args.serving_solves
    reqs = serving.prepare(inputs.serving_stream(n, emax=args.serving_emax), nsteps=100)
    import torch
    budget = 120 << 30
    log("serving inputs ready")
    pool_stats, _ = serving.run_pool(reqs, math.inf, budget)
    torch.cuda.synchronize(dev)
    serial_stats, _ = serving.run_serial(reqs, math.inf)
    # latency at a finite arrival rate: half of the pool's measured capacity
    rate = 0.5 * pool_stats["solves_per_s"]
    pool_rate_stats, _ = serving.run_pool(reqs, rate, budget)
    # and at a quarter of and at the full measured capacity (p50 / p99 against the arrival rate)
    sweep = []
    for frac in (0.25, 1.0):
        st, _ = serving.run_pool(reqs, frac * pool_stats["solves_per_s"], budget)
        sweep.append({"rate_per_s": frac * pool_stats["solves_per_s"], "fraction_of_capacity": frac,
                      "solves_per_s": st["solves_per_s"], "p50_s": st["p50_s"], "p99_s": st["p99_s"]})
    sweep.insert(1, {"rate_per_s": rate, "fraction_of_capacity": 0.5, "solves_per_s": pool_rate_stats["solves_per_s"],
                     "p50_s": pool_rate_stats["p50_s"], "p99_s": pool_rate_stats["p99_s"]})
    # the one-solve-at-a-time FP64 path: every request in FP64, one after another
    reqs = serving.as_fp64(reqs)
    serial64_stats, _ = serving.run_serial(reqs, math.inf)
    del reqs
    return {"workload": f"{n} independent 2D solves (advection / isothermal Euler 50/50, elements per axis "
                        f"log-uniform in [16,{args.serving_emax}], degree in {{3,5,7}}, FP64/FP32 50/50), "
                        "100 RK4 steps each, 120 GB budget",
            "burst": {"pool": pool_stats, "one_at_a_time": serial_stats, "one_at_a_time_all_f64": serial64_stats,
                      "speedup_solves_per_s": pool_stats["solves_per_s"] / serial_stats["solves_per_s"],
                      "speedup_vs_f64_one_at_a_time": pool_stats["solves_per_s"] / serial64_stats["solves_per_s"]},
            "poisson_half_capacity": {"rate_per_s": rate, "pool": pool_rate_stats},
            "poisson_rate_sweep": sweep}


def run_workload_table(dev, peaks):
    """The other full-size problems (2D isothermal Euler 512^2 degree 7, 3D isothermal Euler 64^3
    degree 5, and 32^3 at degree 7): ms per RK4 stage of the autotuned tile in FP64 and FP32, CUDA
    events around a run of RK4 steps, with the FP64-pipe and HBM roofline fractions.  Their working
    sets (>= 0.27 GB per array) are larger than L2."""
    import torch
    from paper_2510_05254_b300 import inputs
    from paper_2510_05254_b300.solver import Solver
    hbm = peaks.get("hbm_gbs", 6400.0)
    p64 = fp64_peak_tflops(peaks.get("sm_max_mhz", 2032.0))
    out = {}
    for name, nsteps in (("euler2d", 25), ("euler3d", 5), ("euler3d7", 5)):
        dim, deg, el, eq, vel, _, desc = WORKLOADS[name]
        row = {"workload": desc}
        U0 = None
        finals = {}
        for dtype in ("f64", "f32"):
            s = Solver(dim, deg, el, equation=eq, velocity=vel, dtype=dtype, device=dev)
            if U0 is None:
                X = s.node_coords()
                U0 = np.ascontiguousarray(inputs.euler_shear(X) if dim == 2 else inputs.taylor_green(X))
                del X
            s.set_state(U0)
            dt = s.stable_dt(CFL)
            epb, _ = s.autotune(RK)
            log(f"{name} {dtype} autotuned (epb {epb})")
            n = nsteps
            s.set_state(U0)  # the autotuner restored it; start the timed run from U0 again
            s.step(dt, 1, RK)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s.stream)
            s.step(dt, n, RK)
            b.record(s.stream)
            b.synchronize()
            ms = a.elapsed_time(b) / (n * STAGES)
            r = {"ms_per_stage": ms, "dof_updates_per_s": s.ndof / (ms * 1e-3), "elems_per_block": epb,
                 "mapping": "line" if s.kernel == 1 else "line_var"}
            if dtype == "f64":
                tf = FLOPS_PER_DOF[name] * s.ndof / (ms * 1e-3) / 1e12
                r.update({"tflops": tf, "frac_fp64_peak": tf / p64})
            else:
                gbs = PASSES_PER_STAGE * 4 * s.ndof / (ms * 1e-3) / 1e9
                r.update({"gbs": gbs, "frac_hbm": gbs / hbm})
            finals[dtype] = s.get_state()
            if name == "euler3d":
                # the sixth-order scheme of Eq. (RK6) on the same problem (7 stages, slopes stored)
                s.set_state(U0)
                s.step(dt, 1, 6)
                a.record(s.stream)
                s.step(dt, 2, 6)
                b.record(s.stream)
                b.synchronize()
                ms6 = a.elapsed_time(b) / (2 * 7)
                r["rk6"] = {"ms_per_stage": ms6, "dof_updates_per_s": s.ndof / (ms6 * 1e-3)}
            row[dtype] = r
            row["dof"] = s.ndof
            s.close()
        row["accuracy_f32_vs_f64"] = dict(rel_err(finals["f32"], finals["f64"]), steps=nsteps + 1)
        del U0, finals
        torch.cuda.empty_cache()
        out[name] = row
    return out


def rel_err(a, ref):
    """Relative L2 and Linf difference of two states (numpy, FP64 arithmetic)."""
    d = np.asarray(a, dtype=np.float64) - np.asarray(ref, dtype=np.float64)
    return {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)),
            "rel_linf": float(np.abs(d).max() / np.abs(ref).max()),
            "max_abs_diff": float(np.abs(d).max()), "max_abs_ref": float(np.abs(ref).max())}


def energy_block(r64, r32, work, t64_ms, t32_ms, rff=None, tff_ms=None):
    out = {}
    for name, r, t in (("f64", r64, t64_ms), ("f32", r32, t32_ms), ("f64_ff", rff, tff_ms)):
        if r is None:
            continue
        p = (r["clocks"] or {}).get("power_w")
        if p:
            out[name] = {"power_w_median": p, "joules_per_dof_update": p * t * 1e-3 / work,
                         "dof_updates_per_joule": work / (p * t * 1e-3)}
    return out or None


def run_ours(args, world, rank, dev, pg):
    import torch
    from paper_2510_05254_b300.solver import Solver
    peaks, peak_kind = load_peaks()
    probe = Solver(DIM, DEGREE, ELEMS, equation=EQ, velocity=VEL, dtype="f64", device=dev)
    X = probe.node_coords()
    probe.close()
    U0 = np.ascontiguousarray(initial_condition(X))
    chosen = set(args.variants.split(","))
    skipped = {"total_ms": float("nan"), "stage_ms": float("nan"), "ndof": None, "clocks": None, "epb": None,
               "kernel": None, "l2_norm": None, "mass": None, "state_bytes": 0, "final": None}
    log("initial condition ready")
    r64 = run_solver_timed("f64", args, dev, pg, U0) if "f64" in chosen else dict(skipped)
    log("f64 timed")
    r32 = run_solver_timed("f32", args, dev, pg, U0) if "f32" in chosen else dict(skipped)
    log("f32 timed")
    rff = run_solver_timed("f64ff", args, dev, pg, U0) if "f64ff" in chosen else dict(skipped)
    log("f64ff timed")
    for r in (r64, r32, rff):
        if r["ndof"] is None:
            r["ndof"] = next(x["ndof"] for x in (r64, r32, rff) if x["ndof"] is not None)
    t64 = max_over_ranks(pg, r64["total_ms"], dev)
    t32 = max_over_ranks(pg, r32["total_ms"], dev)
    tff = max_over_ranks(pg, rff["total_ms"], dev)
    work = r64["ndof"] * STAGES * NSTEPS * args.steps
    value = world * work / (t64 * 1e-3)
    value32 = world * work / (t32 * 1e-3)
    e2e_s, nb = run_e2e(args, dev, U0) if "f64" in chosen else (float("nan"), 0)
    log("e2e timed")
    e2e_s = max_over_ranks(pg, e2e_s, dev)
    # roofline of the dominant kernel (the fused stage kernel)
    clocks = r64["clocks"] or {}
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    p64 = fp64_peak_tflops(peaks.get("sm_max_mhz", 2032.0))
    ach64 = FLOPS_PER_DOF_STAGE * r64["ndof"] / (r64["stage_ms"] * 1e-3) / 1e12
    bytes32 = PASSES_PER_STAGE * 4 * r32["ndof"]
    ach32 = bytes32 / (r32["stage_ms"] * 1e-3) / 1e9
    hbm = peaks.get("hbm_gbs", 6400.0)
    line = {
        "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t64 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": data_description(),
        "config": config_block(world),
        "e2e": {"value": world * work / e2e_s, "unit": "DOF-updates/s", "h2d_bytes_per_step": nb,
                "d2h_bytes_per_step": nb + 8 * 8},
        "gpu_launches": args.steps * (NSTEPS * STAGES + 2),  # per variant timed region
        "roofline": {"bound": "alu", "achieved": ach64, "peak": p64, "unit": "TFLOP/s", "frac": ach64 / p64,
                     "traffic": TRAFFIC_PER_LAUNCH.get((args.workload, "f64")) if not args.elems else None,
                     "traffic_note": "DRAM bytes per stage launch (ncu, mean of the 4 RK4 stages); algorithmic "
                                     "%.1f MB: part of the 4 x %.1f MB arrays stays in L2" % (
                                         PASSES_PER_STAGE * 8 * r64["ndof"] / 1e6, 8 * r64["ndof"] / 1e6),
                     "kernel": f"stage_kernel<{DIM},{DEGREE},{EQ},double>",
                     "peak_note": "FP64 pipe: 148 SMs x 2 DFMA/clk x 2 flop at the max SM clock (derived)",
                     "stage_ms": r64["stage_ms"], "elems_per_block": r64["epb"],
                     "mapping": r64["kernel"]},
        "f32": {"value": value32, "unit": "DOF-updates/s", "ms_per_step": t32 / args.steps,
                "roofline": {"bound": "hbm", "achieved": ach32, "peak": hbm, "unit": "GB/s",
                             "frac": ach32 / hbm,
                             "traffic": TRAFFIC_PER_LAUNCH.get((args.workload, "f32")) if not args.elems else None,
                             "kernel": f"stage_kernel<{DIM},{DEGREE},{EQ},float>",
                             "peak_kind": peak_kind, "stage_ms": r32["stage_ms"],
                             "elems_per_block": r32["epb"], "mapping": r32["kernel"],
                             "note": ("working set 4 x %.1f MB %s the 126 MB L2" % (
                                 r32["state_bytes"] / 1e6,
                                 "fits" if 4 * r32["state_bytes"] < 126e6 else "exceeds"))}},
        # FP64 state and stage update with the D contraction in float-float on the FP32 pipe
        # (NDG_F64_FF): held to the FP64 parity bar (1e-12 relative L2 per step vs the oracle)
        "f64_ff": {"value": world * work / (tff * 1e-3), "unit": "DOF-updates/s", "ms_per_step": tff / args.steps,
                   "stage_ms": rff["stage_ms"], "elems_per_block": rff["epb"], "mapping": rff["kernel"],
                   "parity": "1e-12 relative L2 per step vs the FP64 oracle (tests/test_gpu_parity.py)",
                   "l2_norm": rff["l2_norm"]},
        "clocks": r64["clocks"],
        # energy per DOF-update from the measured board power during the timed region (the paper's
        # energy comparison, Sec. 3.3, multiplies TDP by run time instead)
        "energy": energy_block(r64, r32, work, t64, t32, rff, tff),
        "check": {"l2_norm_f64": r64["l2_norm"], "l2_norm_f32": r32["l2_norm"], "l2_norm_f64_ff": rff["l2_norm"],
                  "mass_f64": r64["mass"]},
        # the FP64 path matches the oracle to 1e-12 per step (tests), so these are the other
        # precisions' errors against the method in FP64 after NSTEPS steps
        "accuracy": {"steps": NSTEPS,
                     "f32_vs_f64": (rel_err(r32["final"], r64["final"])
                                    if r32.get("final") is not None and r64.get("final") is not None else None),
                     "f64_ff_vs_f64": (rel_err(rff["final"], r64["final"])
                                       if rff.get("final") is not None and r64.get("final") is not None else None)},
    }
    if rank == 0 and not args.no_cpu_baseline:
        rate, el = oracle_sample(args.cpu_steps)
        line["cpu_baseline"] = {"value": rate, "unit": "DOF-updates/s", "cores": 1, "kind": "oracle",
                                "sample": f"{args.cpu_steps} RK4 steps of the full 4.19M-DOF workload "
                                          f"({el:.1f} s, single-threaded FP64 oracle)"}
    log("cpu baseline done")
    if not args.no_workloads and args.workload == "adv2d":
        line["workloads"] = run_workload_table(dev, peaks)
        log("workload table done")
    if rank == 0 and not args.no_serving:
        line["serving"] = run_serving(args, dev)
        log("serving done")
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the 2D / 3D isothermal Euler table (FP64 and FP32 ms per stage)")
    ap.add_argument("--cpu-steps", type=int, default=15)
    ap.add_argument("--serving-solves", type=int, default=200)
    ap.add_argument("--serving-emax", type=int, default=512)
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="adv2d")
    ap.add_argument("--epb", type=int, default=0,
                    help="elements per CTA tile instead of autotuning (profiler captures)")
    ap.add_argument("--elems", type=int, default=0,
                    help="elements per axis instead of the workload's (smaller cases for profiler captures)")
    ap.add_argument("--variants", default="f64,f32,f64ff",
                    help="precisions to time (comma list of f64, f32, f64ff); f64 is the headline")
    args = ap.parse_args()
    select_workload(args.workload)
    if args.elems:
        global ELEMS, WORKLOAD
        ELEMS = (args.elems,) * DIM
        WORKLOAD = WORKLOAD.split(",")[0] + f", {args.elems}^{DIM} elements (reduced for a profiler capture)"
        args.no_cpu_baseline = True
        args.no_workloads = True
    global FLOPS_PER_DOF_STAGE
    FLOPS_PER_DOF_STAGE = FLOPS_PER_DOF[args.workload]
    if args.workload != "adv2d":  # the roofline flop count and the CPU sample are the bench workload's
        args.no_cpu_baseline = True
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        line = run_ours(args, world, rank, local, pg)
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
