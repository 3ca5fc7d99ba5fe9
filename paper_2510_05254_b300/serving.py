"""Serving driver: a stream of independent solves arriving as a Poisson process, run either
through the pool (ndg_pool_*: admission under a memory budget + continuous batching) or one at a
time through a single context per solve (create, set_state, step, get_state, destroy).

Latency = time the result is on the host - arrival time; throughput = solves / (last completion -
first arrival).  All computation is libndg's; this module only schedules submissions.
"""
from __future__ import annotations

import math
import threading
import time

import numpy as np

from . import inputs
from . import native as nat

CFL = 0.1


def prepare(requests, nsteps=100):
    """Initial states and time steps of the serving workload (outside any timed region).  The node
    coordinates come from the library (ndg_node_coords: the 1D coordinates along x of one row of
    elements, the same along y), the initial conditions from their separable grid forms (the same
    values as the pointwise ones), and the time step from the library's CFL rule applied to that
    state (ndg_stable_dt)."""
    import torch
    out = []
    x_of = {}
    ctx_of = {}
    try:
        for r in requests:
            E, N = r["elems"], r["degree"]
            cfg = _cfg(r)
            cfg.stream = torch.cuda.current_stream().cuda_stream
            key = (E, N, r["equation"], r["dtype"])
            if key not in ctx_of:
                ctx_of[key] = nat.ndg_create_ex(cfg)
            ctx = ctx_of[key]
            if (E, N) not in x_of:
                info = nat.ndg_info(ctx)
                X = np.empty((2, info.nelem, info.nodes_per_elem))
                nat.ndg_node_coords(ctx, X.ctypes.data, X.size)
                x_of[(E, N)] = np.ascontiguousarray(X[0, :E, :N + 1]).reshape(-1)  # row ey = 0, j = 0
            kind = "gaussian_noise" if r["equation"] == 0 else "euler_shear"
            U = inputs.grid_state(kind, x_of[(E, N)], E, N + 1, r["seed"])
            U = np.ascontiguousarray(U, dtype=np.float64 if r["dtype"] == "f64" else np.float32)
            nat.ndg_set_state(ctx, U.ctypes.data, U.nbytes, False)
            dt = nat.ndg_stable_dt(ctx, CFL)
            out.append(dict(r, U=U, dt=dt, nsteps=nsteps))
            if len(ctx_of) > 8:  # keep few contexts (and their device memory) alive
                for k in [k for k in ctx_of if k != key]:
                    nat.ndg_destroy(ctx_of.pop(k))
    finally:
        for c in ctx_of.values():
            nat.ndg_destroy(c)
    return out


def as_fp64(reqs):
    """The same requests, every one in FP64 (states widened in place of a new draw)."""
    return [dict(r, dtype="f64", U=np.ascontiguousarray(r["U"], dtype=np.float64)) for r in reqs]


def _cfg(r):
    cfg = nat.ndg_config_init()
    cfg.dim, cfg.degree = 2, r["degree"]
    cfg.elems[0] = cfg.elems[1] = r["elems"]
    cfg.equation = r["equation"]
    cfg.flux = nat.NDG_FLUX_UPWIND if r["equation"] == 0 else nat.NDG_FLUX_LLF
    cfg.velocity[0], cfg.velocity[1] = 1.0, 0.5
    cfg.dtype = nat.NDG_F64 if r["dtype"] == "f64" else nat.NDG_F32
    return cfg


def _stats(lat, t_first, t_last, n):
    lat = np.sort(np.asarray(lat))
    return {"solves": n, "solves_per_s": n / max(t_last - t_first, 1e-9),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "wall_s": t_last - t_first}


def run_pool(reqs, rate: float, budget_bytes: int, keep_results: bool = False):
    """Submit at Poisson arrival times (rate solves/s; inf = all at once) and wait for all."""
    pool = nat.ndg_pool_create(budget_bytes)
    arrivals = _arrivals(reqs, rate)
    tickets = [None] * len(reqs)
    results = [None] * len(reqs)

    def submitter():
        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            wait = arrivals[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets[i] = nat.ndg_pool_submit(pool, _cfg(r), r["U"].ctypes.data, r["U"].nbytes, 4, r["dt"],
                                             r["nsteps"])

    try:
        th = threading.Thread(target=submitter)
        th.start()
        lat, first, last = [], math.inf, 0.0
        for i, r in enumerate(reqs):
            while tickets[i] is None:
                time.sleep(1e-4)
            out = np.empty_like(r["U"]) if keep_results else None
            rc, st = nat.ndg_pool_poll(pool, tickets[i], out.ctypes.data if out is not None else None,
                                       r["U"].nbytes if out is not None else 0, 3600.0)
            assert rc == nat.NDG_OK
            results[i] = out
            lat.append(st.latency_s)
            first, last = min(first, st.submit_s), max(last, st.done_s)
        th.join()
        status = nat.ndg_pool_status(pool)
    finally:
        nat.ndg_pool_destroy(pool)
    s = _stats(lat, first, last, len(reqs))
    s["peak_bytes"] = status["peak_bytes"]
    s["budget_bytes"] = budget_bytes
    return s, results


def run_serial(reqs, rate: float, keep_results: bool = False):
    """One solve at a time, in arrival order, each through its own context."""
    import torch
    arrivals = _arrivals(reqs, rate)
    t0 = time.perf_counter()
    lat, results = [], []
    done_last = 0.0
    for i, r in enumerate(reqs):
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        cfg = _cfg(r)
        cfg.stream = torch.cuda.current_stream().cuda_stream
        ctx = nat.ndg_create_ex(cfg)
        try:
            nat.ndg_set_state(ctx, r["U"].ctypes.data, r["U"].nbytes, False)
            nat.ndg_step(ctx, r["dt"], r["nsteps"], 4)
            out = np.empty_like(r["U"])
            nat.ndg_get_state(ctx, out.ctypes.data, out.nbytes, False)
        finally:
            nat.ndg_destroy(ctx)
        done = time.perf_counter() - t0
        lat.append(done - arrivals[i])
        done_last = done
        results.append(out if keep_results else None)
    return _stats(lat, 0.0, done_last, len(reqs)), results


def _arrivals(reqs, rate):
    if not math.isfinite(rate):
        return [0.0] * len(reqs)
    t, out = 0.0, []
    for r in reqs:
        t += r["gap"] / rate
        out.append(t)
    return out
