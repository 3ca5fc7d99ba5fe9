"""Benchmark of the NDG + RK hot path on B300: DOF-updates per second per RK stage.

Headline workload (one bench step): the 3D isothermal Euler problem of the paper's Sec. 3.2 at
degree 5 -- 64^3 hexahedral elements of 6^3 LGL nodes, 4 x 384^3 = 226.5M DOF, rho = 1 and a
Taylor-Green velocity of amplitude 0.1, local Lax-Friedrichs flux, classical RK4 at CFL 0.1 --
advanced 10 RK4 steps (40 launches of the fused stage kernel) from its initial state, followed by
the norms reduction.  The state is reset from a device-resident copy at the start of every bench
step; every array (1.8 GB in FP64) is far larger than the 126 MB L2.  FP64 is the headline, FP32
is reported beside it.  The line also carries: the same workload end to end through the C ABI
with host buffers (`e2e`), the oracle on the host's cores (`cpu_baseline`), a table of the other
problems (2D advection 256^2 and 2D isothermal Euler 512^2 at degree 7, 3D isothermal Euler
32^3 at degree 7, and this one), each timed for at least 2.5 s with board power sampled (energy
per DOF-update), and the serving stream (pool versus one solve at a time, Poisson arrivals at
multiples of the one-at-a-time FP64 capacity).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-serving]
                    [--no-workloads] [--no-cpu-baseline] [--serving-solves S] [--serving-sweep-solves S]
                    [--serving-only] [--workload euler3d|adv2d|euler2d|euler3d7] [--elems E] [--epb T]
                    [--variants f64,f32,f64ff]

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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RK stage (FP64 vs FP32); batched solves/s + p50/p99 latency"
# name: (dim, degree, elements, equation, velocity, RK4 steps per bench step, description)
WORKLOADS = {
    "euler3d": (3, 5, (64, 64, 64), 1, (0.0, 0.0, 0.0), 10,
                "3D isothermal Euler, 64^3 elements, degree 5 (6^3 LGL nodes), 4 x 384^3 = 226.5M DOF, "
                "Taylor-Green velocity amplitude 0.1, LLF flux, RK4 at CFL 0.1"),
    "adv2d": (2, 7, (256, 256), 0, (1.0, 0.5, 0.0), 1000,
              "2D linear advection, 256^2 elements, degree 7 (8^2 LGL nodes), 2048^2 = 4.19M DOF, "
              "velocity (1, 0.5), upwind flux, RK4 at CFL 0.1"),
    "euler2d": (2, 7, (512, 512), 1, (0.0, 0.0, 0.0), 200,
                "2D isothermal Euler, 512^2 elements, degree 7, 3 x 4096^2 = 50.3M DOF, LLF flux, RK4 at CFL 0.1"),
    # the eighth-order 3D case (degree 7) at the same size class
    "euler3d7": (3, 7, (32, 32, 32), 1, (0.0, 0.0, 0.0), 50,
                 "3D isothermal Euler, 32^3 elements, degree 7 (8^3 LGL nodes), 4 x 256^3 = 67.1M DOF, "
                 "LLF flux, RK4 at CFL 0.1"),
}
HEADLINE = "euler3d"
DIM, DEGREE, ELEMS, EQ, VEL, NSTEPS, WORKLOAD = WORKLOADS[HEADLINE]
CFL, RK = 0.1, 4
STAGES = 4
PASSES_PER_STAGE = 4.0  # RK4 array passes per stage: 3, 5, 5, 3
# Algorithmic FP64 work of one RK4 stage per DOF (sum-factorised strong-form volume term d axes x
# n FMA, per-axis scaling, lifted face terms, stage update averaged over the four stages): 2D
# advection degree 7: 40 flop; 2D isothermal Euler degree 7: 48; 3D isothermal Euler degree 5:
# 60; degree 7: 72 (the volume term 3 axes x 8 FMA = 48 instead of 3 x 6 = 36).
FLOPS_PER_DOF = {"adv2d": 40.0, "euler2d": 48.0, "euler3d": 60.0, "euler3d7": 72.0}
# DRAM bytes (read + write) per stage launch of the headline's kernels, mean of the four RK4
# stages, from ncu captures of dram__bytes_read.sum + dram__bytes_write.sum at 48^3 elements
# scaled to 64^3 by the DOF count (commands and per-stage values in
# profiles/stage_kernel_euler3d_deg5_64cubed.md).  The figures hold for the kernel sources they
# were captured from: TRAFFIC_SOURCES_SHA1 is the digest of those files at the capture, and a
# bench run whose sources differ reports traffic null until the capture is repeated.
TRAFFIC_PER_LAUNCH = {("euler3d", "f64"): 7.3277e9, ("euler3d", "f32"): 3.5670e9}
TRAFFIC_SOURCES = ["stage_kernel.cuh", "stage_euler3d_f32.cuh", "stage_dispatch.cuh", "stage_f64_d3.cu",
                   "stage_f32_d3.cu", "ndg_internal.h"]
TRAFFIC_SOURCES_SHA1 = "9e49c7a5c650fb41a76f9e894a72a9f852da81b9"


def kernel_sources_sha1():
    """SHA-1 of the kernel sources' code: line comments, trailing blanks and empty lines removed
    (the files hold no '//' inside string literals), so that a comment edit keeps the capture."""
    import hashlib
    import re
    h = hashlib.sha1()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2510_05254_b300", "csrc", name)) as f:
            for line in f:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def traffic_per_launch(workload, dtype, reduced):
    """The captured DRAM bytes per launch, or None (a reduced problem, no capture for this
    workload, or kernel sources changed since the capture)."""
    if reduced or kernel_sources_sha1() != TRAFFIC_SOURCES_SHA1:
        return None
    return TRAFFIC_PER_LAUNCH.get((workload, dtype))


L2_BYTES = 126e6

_T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    sys.stderr.write(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}\n")
    sys.stderr.flush()


def select_workload(name):
    global DIM, DEGREE, ELEMS, EQ, VEL, NSTEPS, WORKLOAD
    DIM, DEGREE, ELEMS, EQ, VEL, NSTEPS, WORKLOAD = WORKLOADS[name]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def fp64_peak_tflops(sm_mhz):
    # 148 SMs x 2 DFMA / clock / SM x 2 flop (B300 FP64 units; 1.12 TFLOP/s measured at 1935 MHz)
    return 148 * 2 * 2 * sm_mhz * 1e6 / 1e12


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clocks / throttle reasons / board power sampled every 200 ms during a timed
    region."""

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


def data_description(eq=None, dim=None):
    eq = EQ if eq is None else eq
    dim = DIM if dim is None else dim
    if eq == 0:
        return "synthetic (seeded Gaussian pulse + Fourier noise)"
    if dim == 2:
        return "synthetic (isothermal Euler: density 1 + 0.1 sin sin, seeded smooth shear velocity, Mach <= 0.3)"
    return "synthetic (isothermal Euler: density 1, Taylor-Green velocity of amplitude 0.1)"


def initial_condition(X, eq=None, dim=None):
    from paper_2510_05254_b300 import inputs
    eq = EQ if eq is None else eq
    dim = DIM if dim is None else dim
    if eq == 0:
        return inputs.gaussian_noise(X)
    return inputs.euler_shear(X) if dim == 2 else inputs.taylor_green(X)


def ndof_of(dim, degree, elems, eq):
    return (1 if eq == 0 else dim + 1) * int(np.prod(elems)) * (degree + 1) ** dim


def config_block(world):
    return {"workload": WORKLOAD, "elements": list(ELEMS), "degree": DEGREE, "dof": ndof_of(DIM, DEGREE, ELEMS, EQ),
            "rk_steps_per_bench_step": NSTEPS, "rk_scheme": "RK4 (Eq. (RK4))", "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2: every state array exceeds the 126 MB L2 "
                  f"({ndof_of(DIM, DEGREE, ELEMS, EQ) * 8 / 1e9:.2f} GB in FP64)"}


# ---------------------------------------------------------------------------------------------
# CPU: the oracle (test infrastructure) timed on the host's cores
# ---------------------------------------------------------------------------------------------

def _oracle_problem(elems):
    from oracle import oracle as orc
    return orc.Problem(dim=DIM, degree=DEGREE, elems=tuple(elems) + (1,) * (3 - DIM), equation=EQ, flux=EQ,
                       velocity=VEL)


def oracle_rate(elems, threads, min_seconds):
    """DOF-updates/s per RK4 stage of the oracle's -O3 -march=native build on `elems` elements of
    the workload's problem, split over `threads` threads (1: orc_step itself); RK4 steps are
    repeated until min_seconds have passed.  Returns (rate, seconds, steps)."""
    from oracle import oracle as orc
    p = _oracle_problem(elems)
    U0 = initial_condition(orc.node_coords(p))
    dt = orc.stable_dt(p, U0, CFL)

    def one():
        if threads > 1:
            return orc.step_threads(p, U0, dt, 1, RK, threads=threads, native=True)
        return orc.step_native(p, U0, dt, 1, RK)

    one()  # first touch of the buffers, library load
    steps, el = 0, 0.0
    while el < min_seconds or steps < 1:
        t = time.perf_counter()
        one()
        el += time.perf_counter() - t
        steps += 1
    return p.ndof * STAGES * steps / el, el, steps


def cpu_sample_elems():
    """Reduced grids of the workload for the CPU samples: all cores on 1/8 of the elements, one
    thread on 1/64 (3D) -- the oracle needs 10 state-sized host arrays."""
    if DIM == 3:
        return tuple(max(2, e // 2) for e in ELEMS), tuple(max(2, e // 4) for e in ELEMS)
    return tuple(max(2, e // 2) for e in ELEMS), tuple(max(2, e // 4) for e in ELEMS)


def cpu_baseline_block():
    cores = host_cores()
    many, one = cpu_sample_elems()
    rate_mt, el_mt, st_mt = oracle_rate(many, cores, 8.0)
    rate_1, el_1, st_1 = oracle_rate(one, 1, 8.0)
    ndof_mt, ndof_1 = ndof_of(DIM, DEGREE, many, EQ), ndof_of(DIM, DEGREE, one, EQ)
    return {"value": rate_mt, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{st_mt} RK4 step(s) of the workload's problem on {'x'.join(map(str, many))} elements "
                      f"({ndof_mt / 1e6:.1f}M DOF) in {el_mt:.1f} s, the oracle's -O3 -march=native build split "
                      f"by element ranges over {cores} threads (orc_step_threads, bitwise equal to one thread)",
            "single_thread": {"value": rate_1, "unit": "DOF-updates/s", "cores": 1,
                              "sample": f"{st_1} RK4 step(s) on {'x'.join(map(str, one))} elements "
                                        f"({ndof_1 / 1e6:.2f}M DOF) in {el_1:.1f} s, orc_step, -O3 -march=native"}}


def run_reference(args, world, rank):
    """The oracle as it stands, on the machine's host cores, for the same metric and workload: each
    bench step one RK4 step of the workload's problem on 1/8 of its elements (all cores)."""
    if rank != 0:
        return None
    from oracle import oracle as orc
    cores = host_cores()
    many, _ = cpu_sample_elems()
    p = _oracle_problem(many)
    U0 = initial_condition(orc.node_coords(p))
    dt = orc.stable_dt(p, U0, CFL)
    for _ in range(args.warmup):
        orc.step_threads(p, U0, dt, 1, RK, threads=cores, native=True)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        orc.step_threads(p, U0, dt, 1, RK, threads=cores, native=True)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = p.ndof * STAGES * args.steps / tot
    sample = (f"1 RK4 step per bench step of the workload's problem on {'x'.join(map(str, many))} elements "
              f"({p.ndof / 1e6:.1f}M DOF, 1/8 of the workload's elements), the oracle's -O3 -march=native build "
              f"split by element ranges over {cores} threads")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": data_description(), "config": config_block(world),
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------------------------
# GPU: the headline workload
# ---------------------------------------------------------------------------------------------

def run_solver_timed(dtype, args, dev, pg, U0_host):
    """Device-timed bench steps of one precision: per-step device ms, stage-kernel ms, clocks."""
    import torch
    from paper_2510_05254_b300 import native as nat
    from paper_2510_05254_b300.solver import Solver
    s = Solver(DIM, DEGREE, ELEMS, equation=EQ, velocity=VEL, dtype=dtype, device=dev,
               elems_per_block=args.epb)
    U0 = torch.tensor(U0_host, device=f"cuda:{dev}", dtype=s.torch_dtype)
    s.set_state(U0)
    dt = s.stable_dt(CFL)
    epb = args.epb or s.autotune(RK)[0]  # the library's tile autotuner (state restored bitwise)

    def one(evs=None):
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
           "kernel": "line" if s.kernel == 1 else "line_var", "l2_norm": nr.l2, "mass": nr.integral[0],
           "state_bytes": s.state_bytes, "final": s.get_state()}
    s.close()
    return out


def run_e2e(args, dev, U0_host):
    """The same bench step through the C ABI with HOST buffers: a pinned host-to-device copy of the
    initial state, NSTEPS RK4 steps, a device-to-host copy of the final state and of the norms.
    Two contexts, each on its own stream, take the bench steps in turn: the host issues step k+1's
    upload and RK steps before it waits for step k's download, so one step's copies overlap the
    other's RK steps (a throughput pipeline; every step still moves its own bytes both ways)."""
    import torch
    from paper_2510_05254_b300 import native as nat
    from paper_2510_05254_b300.solver import Solver
    ctxs = [Solver(DIM, DEGREE, ELEMS, equation=EQ, velocity=VEL, dtype="f64", device=dev, elems_per_block=args.epb)
            for _ in range(2)]
    src = torch.from_numpy(np.ascontiguousarray(U0_host, dtype=np.float64)).pin_memory()
    dsts = [torch.empty_like(src).pin_memory() for _ in ctxs]
    nat.ndg_set_state(ctxs[0].ctx, src.data_ptr(), ctxs[0].state_bytes, False)
    dt = ctxs[0].stable_dt(CFL)

    def issue(k):
        c = ctxs[k % 2]
        nat.ndg_set_state(c.ctx, src.data_ptr(), c.state_bytes, False)
        nat.ndg_step(c.ctx, dt, NSTEPS, RK)

    def finish(k):
        c = ctxs[k % 2]
        nat.ndg_get_state(c.ctx, dsts[k % 2].data_ptr(), c.state_bytes, False)
        return nat.ndg_norms(c.ctx)

    def run(n):
        issue(0)
        for k in range(n):
            if k + 1 < n:
                issue(k + 1)
            finish(k)

    run(max(2, args.warmup))
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    run(args.steps)
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t
    nb = ctxs[0].state_bytes
    # the same input gives the same result in either context
    same = args.steps < 2 or bool(torch.equal(dsts[0], dsts[1]))
    for c in ctxs:
        c.close()
    if not same:
        raise RuntimeError("end-to-end: the two contexts returned different states for the same input")
    return el, nb


# ---------------------------------------------------------------------------------------------
# the table of problems: ms per stage, roofline fractions and energy per DOF-update
# ---------------------------------------------------------------------------------------------

def timed_row(name, dtype, dev, peaks, U0, min_seconds=2.5):
    """One problem in one precision: autotuned tile, RK4 steps timed with CUDA events for at least
    min_seconds with board power sampled throughout."""
    import torch
    from paper_2510_05254_b300.solver import Solver
    dim, deg, el, eq, vel, _, desc = WORKLOADS[name]
    s = Solver(dim, deg, el, equation=eq, velocity=vel, dtype=dtype, device=dev)
    s.set_state(U0)
    dt = s.stable_dt(CFL)
    epb, _ = s.autotune(RK)
    s.set_state(U0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s.stream)
    s.step(dt, 2, RK)
    b.record(s.stream)
    b.synchronize()
    per_step = a.elapsed_time(b) / 2
    n = max(4, int(math.ceil(min_seconds * 1e3 / per_step)))
    s.set_state(U0)
    with ClockSampler(dev) as clk:
        a.record(s.stream)
        s.step(dt, n, RK)
        b.record(s.stream)
        b.synchronize()
    ms = a.elapsed_time(b) / (n * STAGES)
    r = {"ms_per_stage": ms, "dof_updates_per_s": s.ndof / (ms * 1e-3), "elems_per_block": epb,
         "mapping": "line" if s.kernel == 1 else "line_var", "timed_rk4_steps": n,
         "timed_s": a.elapsed_time(b) * 1e-3}
    hbm = peaks.get("hbm_gbs", 6400.0)
    if dtype == "f32":
        gbs = PASSES_PER_STAGE * 4 * s.ndof / (ms * 1e-3) / 1e9
        r.update({"gbs": gbs, "frac_hbm": gbs / hbm})
    else:
        tf = FLOPS_PER_DOF[name] * s.ndof / (ms * 1e-3) / 1e12
        r.update({"tflops": tf, "frac_fp64_peak": tf / fp64_peak_tflops(peaks.get("sm_max_mhz", 2032.0))})
    c = clk.summary() or {}
    if c.get("power_w"):
        work = s.ndof * STAGES * n
        r["energy"] = {"power_w_median": c["power_w"], "power_samples": c["samples"],
                       "joules_per_dof_update": c["power_w"] * r["timed_s"] / work,
                       "dof_updates_per_joule": work / (c["power_w"] * r["timed_s"])}
    r["clocks"] = {k: c.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    final = s.get_state()
    s.close()
    return r, final, n, dt


def run_workload_table(dev, peaks, names):
    import torch
    from paper_2510_05254_b300.solver import Solver
    out = {}
    for name in names:
        dim, deg, el, eq, vel, _, desc = WORKLOADS[name]
        probe = Solver(dim, deg, el, equation=eq, velocity=vel, dtype="f64", device=dev)
        X = probe.node_coords()
        probe.close()
        U0 = np.ascontiguousarray(initial_condition(X, eq, dim))
        del X
        row = {"workload": desc, "dof": ndof_of(dim, deg, el, eq)}
        finals = {}
        for dtype in ("f64", "f32", "f64ff"):
            r, final, n, dt = timed_row(name, dtype, dev, peaks, U0)
            row[dtype] = r
            log(f"{name} {dtype}: {r['ms_per_stage']:.4f} ms per stage ({n} RK4 steps)")
            # the accuracy of the other precisions against FP64 after the same first steps
            finals[dtype] = final
        row["accuracy_vs_f64"] = {"note": "each precision's state after its own timed run compared with the FP64 "
                                          "state after its timed run: meaningful only when the step counts agree"}
        for dtype in finals:
            if dtype != "f64" and row[dtype]["timed_rk4_steps"] == row["f64"]["timed_rk4_steps"]:
                row["accuracy_vs_f64"][dtype] = rel_err(finals[dtype], finals["f64"])
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


# ---------------------------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------------------------

def run_serving(args, dev):
    """The serving stream: a burst (all arrivals at once) through the pool, one solve at a time
    with the same dtypes, and one FP64 solve at a time; the same for the solves whose working set
    fits in L2; then Poisson arrivals at 0.25 to 4 times the one-at-a-time FP64 capacity."""
    import torch
    from paper_2510_05254_b300 import inputs, serving
    n = args.serving_solves
    budget = 120 << 30
    reqs = serving.prepare(inputs.serving_stream(n, emax=args.serving_emax), nsteps=100)
    log(f"serving inputs ready ({n} solves)")
    pool_stats, _ = serving.run_pool(reqs, math.inf, budget)
    torch.cuda.synchronize(dev)
    serial_stats, _ = serving.run_serial(reqs, math.inf)
    reqs64 = serving.as_fp64(reqs)
    serial64_stats, _ = serving.run_serial(reqs64, math.inf)
    del reqs64
    log("serving bursts done")
    # the sub-L2 solves (working set of the four RK4 arrays below the 126 MB L2)
    small = [r for r in reqs if 4 * r["U"].nbytes < L2_BYTES]
    small_block = None
    if small:
        ps, _ = serving.run_pool(small, math.inf, budget)
        ss, _ = serving.run_serial(small, math.inf)
        s64, _ = serving.run_serial(serving.as_fp64(small), math.inf)
        small_block = {"solves": len(small), "pool": ps, "one_at_a_time": ss, "one_at_a_time_all_f64": s64,
                       "speedup_solves_per_s": ps["solves_per_s"] / ss["solves_per_s"],
                       "speedup_vs_f64_one_at_a_time": ps["solves_per_s"] / s64["solves_per_s"]}
    # Poisson arrivals at multiples of the one-at-a-time FP64 capacity
    cap64 = serial64_stats["solves_per_s"]
    sweep_reqs = reqs[:args.serving_sweep_solves]
    sweep = []
    for frac in (0.25, 0.5, 1.0, 2.0, 4.0):
        st, _ = serving.run_pool(sweep_reqs, frac * cap64, budget)
        sweep.append({"rate_per_s": frac * cap64, "multiple_of_f64_one_at_a_time_capacity": frac,
                      "solves": len(sweep_reqs), "solves_per_s": st["solves_per_s"], "p50_s": st["p50_s"],
                      "p99_s": st["p99_s"]})
        log(f"serving sweep {frac}x done")
    del reqs
    return {"workload": f"{n} independent 2D solves (advection / isothermal Euler 50/50, elements per axis "
                        f"log-uniform in [16,{args.serving_emax}], degree in {{3,5,7}}, FP64/FP32 50/50), "
                        "100 RK4 steps each, 120 GB budget",
            "burst": {"pool": pool_stats, "one_at_a_time": serial_stats, "one_at_a_time_all_f64": serial64_stats,
                      "speedup_solves_per_s": pool_stats["solves_per_s"] / serial_stats["solves_per_s"],
                      "speedup_vs_f64_one_at_a_time": pool_stats["solves_per_s"] / serial64_stats["solves_per_s"]},
            "burst_sub_l2_solves": small_block,
            "poisson_rate_sweep": sweep,
            "accuracy": "each pool result equals its solve alone bit for bit (tests/test_gpu_serving.py); FP32 "
                        "solves within the FP32 tolerance of the FP64 path"}


# ---------------------------------------------------------------------------------------------

def run_ours(args, world, rank, dev, pg):
    import torch
    from paper_2510_05254_b300.solver import Solver
    peaks, peak_kind = load_peaks()
    line = {}
    if args.serving_only:
        return {"serving": run_serving(args, dev)}
    probe = Solver(DIM, DEGREE, ELEMS, equation=EQ, velocity=VEL, dtype="f64", device=dev)
    X = probe.node_coords()
    probe.close()
    U0 = np.ascontiguousarray(initial_condition(X))
    del X
    chosen = set(args.variants.split(","))
    log("initial condition ready")
    r64 = run_solver_timed("f64", args, dev, pg, U0)
    log(f"f64 timed: {r64['stage_ms']:.4f} ms per stage")
    r32 = run_solver_timed("f32", args, dev, pg, U0) if "f32" in chosen else None
    if r32:
        log(f"f32 timed: {r32['stage_ms']:.4f} ms per stage")
    rff = run_solver_timed("f64ff", args, dev, pg, U0) if "f64ff" in chosen else None
    t64 = max_over_ranks(pg, r64["total_ms"], dev)
    work = r64["ndof"] * STAGES * NSTEPS * args.steps
    value = world * work / (t64 * 1e-3)
    e2e_s, nb = run_e2e(args, dev, U0)
    e2e_s = max_over_ranks(pg, e2e_s, dev)
    log("e2e timed")
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    p64 = fp64_peak_tflops(sm_max)
    flops = FLOPS_PER_DOF[args.workload]
    ach64 = flops * r64["ndof"] / (r64["stage_ms"] * 1e-3) / 1e12
    hbm = peaks.get("hbm_gbs", 6400.0)
    traffic64 = traffic_per_launch(args.workload, "f64", bool(args.elems))
    line.update({
        "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t64 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": data_description(), "config": config_block(world),
        "e2e": {"value": world * work / e2e_s, "unit": "DOF-updates/s", "h2d_bytes_per_step": nb,
                "d2h_bytes_per_step": nb + 8 * 8,
                "note": "per bench step: pinned host->device copy of the initial state, the RK4 steps, "
                        "device->host copy of the final state and of the norms (ndg_set_state / ndg_step / "
                        "ndg_get_state / ndg_norms with host buffers); two contexts on their own streams take "
                        "the steps in turn, so one step's copies overlap the other's RK steps"},
        # kernels of the timed region: NSTEPS x 4 stage launches + 2 norms kernels per bench step
        "gpu_launches": args.steps * (NSTEPS * STAGES + 2),
        "roofline": {"bound": "alu", "achieved": ach64, "peak": p64, "unit": "TFLOP/s", "frac": ach64 / p64,
                     "traffic": traffic64,
                     "traffic_note": "DRAM bytes per stage launch, mean of the four RK4 stages (ncu at 48^3 "
                                     "scaled to 64^3 by the DOF count; null when the kernel sources differ from "
                                     "the captured ones or the problem is reduced); algorithmic %.0f MB (4 array "
                                     "passes x %.0f MB)" % (PASSES_PER_STAGE * 8 * r64["ndof"] / 1e6,
                                                            8 * r64["ndof"] / 1e6),
                     "kernel_sources_sha1": kernel_sources_sha1(),
                     "kernel": f"stage_kernel<{DIM},{DEGREE},{EQ},double>",
                     "flop_per_dof": flops,
                     "peak_note": "FP64 pipe: 148 SMs x 2 DFMA/clk x 2 flop at the max SM clock (derived; "
                                  "1.12 TFLOP/s measured by an FMA-chain probe at 1935 MHz)",
                     "stage_ms": r64["stage_ms"], "elems_per_block": r64["epb"], "mapping": r64["kernel"]},
        "clocks": r64["clocks"],
    })
    if r32:
        t32 = max_over_ranks(pg, r32["total_ms"], dev)
        ach32 = PASSES_PER_STAGE * 4 * r32["ndof"] / (r32["stage_ms"] * 1e-3) / 1e9
        line["f32"] = {"value": world * work / (t32 * 1e-3), "unit": "DOF-updates/s", "ms_per_step": t32 / args.steps,
                       "roofline": {"bound": "hbm", "achieved": ach32, "peak": hbm, "unit": "GB/s",
                                    "frac": ach32 / hbm, "peak_kind": peak_kind,
                                    "traffic": traffic_per_launch(args.workload, "f32", bool(args.elems)),
                                    "kernel": f"stage_kernel_r96<{DIM},{DEGREE},{EQ},float> "
                                              "(euler3d_f32_body)" if DIM == 3 and EQ == 1 else
                                              f"stage_kernel<{DIM},{DEGREE},{EQ},float>",
                                    "stage_ms": r32["stage_ms"], "elems_per_block": r32["epb"],
                                    "mapping": r32["kernel"],
                                    "bytes_per_dof": "4 array passes x 4 B (RK4 passes per stage 3, 5, 5, 3)"},
                       "clocks": r32["clocks"],
                       "accuracy_vs_f64": rel_err(r32["final"], r64["final"])}
    if rff:
        tff = max_over_ranks(pg, rff["total_ms"], dev)
        achff = flops * rff["ndof"] / (rff["stage_ms"] * 1e-3) / 1e12
        line["f64_ff"] = {"value": world * work / (tff * 1e-3), "unit": "DOF-updates/s", "stage_ms": rff["stage_ms"],
                          "elems_per_block": rff["epb"], "mapping": rff["kernel"],
                          "fp64_equivalent_tflops": achff, "frac_fp64_peak": achff / p64,
                          "note": "FP64 state, fluxes and update; the D contraction in float-float (FP32 pipe)",
                          "parity": "1e-12 relative L2 per step vs the FP64 oracle (tests/test_gpu_parity.py)",
                          "accuracy_vs_f64": rel_err(rff["final"], r64["final"])}
    # energy per DOF-update from the board power sampled during the timed region (the paper's
    # energy comparison, Sec. 3.3, multiplies TDP by run time instead)
    energy = {}
    for name, r, t in (("f64", r64, t64), ("f32", r32, None)):
        if r is None or not (r["clocks"] or {}).get("power_w"):
            continue
        t = r["total_ms"] if t is None else t
        energy[name] = {"power_w_median": r["clocks"]["power_w"], "power_samples": r["clocks"]["samples"],
                        "timed_s": t * 1e-3, "joules_per_dof_update": r["clocks"]["power_w"] * t * 1e-3 / work}
    line["energy"] = energy or None
    line["check"] = {"l2_norm_f64": r64["l2_norm"], "mass_f64": r64["mass"],
                     "l2_norm_f32": r32["l2_norm"] if r32 else None}
    del U0, r64, r32, rff
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_block()
        log("cpu baseline done")
    if not args.no_workloads and rank == 0:
        names = [n for n in ("adv2d", "euler2d", "euler3d7", "euler3d") if n in WORKLOADS]
        line["workloads"] = run_workload_table(dev, peaks, names)
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
                    help="skip the table of problems (ms per stage, roofline fractions, energy)")
    ap.add_argument("--serving-solves", type=int, default=200)
    ap.add_argument("--serving-sweep-solves", type=int, default=60,
                    help="solves per Poisson rate of the sweep (the first ones of the stream)")
    ap.add_argument("--serving-emax", type=int, default=512)
    ap.add_argument("--serving-only", action="store_true", help="only the serving block (full-size stream runs)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=HEADLINE)
    ap.add_argument("--epb", type=int, default=0,
                    help="elements per CTA tile instead of autotuning (profiler captures)")
    ap.add_argument("--elems", type=int, default=0,
                    help="elements per axis instead of the workload's (smaller cases for profiler captures)")
    ap.add_argument("--variants", default="f64,f32,f64ff",
                    help="precisions to time beside the FP64 headline (comma list of f32, f64ff)")
    args = ap.parse_args()
    select_workload(args.workload)
    if args.elems:
        global ELEMS, WORKLOAD
        ELEMS = (args.elems,) * DIM
        WORKLOAD = WORKLOAD.split(",")[0] + f", {args.elems}^{DIM} elements (reduced for a profiler capture)"
        args.no_cpu_baseline = True
        args.no_workloads = True
        args.no_serving = True
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
