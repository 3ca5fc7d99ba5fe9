"""Convergence and efficiency studies of the paper's Sec. 3.1, run on the GPU path.

All runs advect the random-mode initial condition of Eq. (initialCond),
U0 = sum_{k=1}^{Nk} A_k sin(2 pi k x) (Nk = 40, A_k ~ U[0,1), y-independent in 2D as printed), with
a = (1, 0, 0) for exactly one revolution (T = 1), so the exact solution is U0 and the error is
the L2 norm of U(T) - U0 (LGL quadrature).  Studies:
  orders      1D, degrees 2..7 (orders 3..8), element counts doubling, RK6 at CFL 0.2: observed
              convergence rate ~ order, and the DOF needed for a 1 % error per order, with the
              Kreiss-Oliger estimate DOF = c (1/error)^(1/order) (c = 200 as in the paper) beside it;
  rk          1D, degree 5, RK3 / RK4 / RK6: the temporal order caps the rate as the grid is refined;
  time2d      2D, degrees 2..7, RK6: error against GPU time (events) -- the paper's error-vs-time view;
  rk_time2d   2D, degree 7, RK3 / RK4 / RK6: error against GPU time.

    python -m paper_2510_05254_b300.studies [orders rk time2d rk_time2d] [--out file.json]
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np

from . import inputs
from . import native as nat

NK = 40


def run_case(dim: int, degree: int, elems: int, rk: int, cfl: float, dtype: str = "f64",
             seed: int = inputs.BASE_SEED) -> dict:
    """One revolution of the random-mode profile; returns DOF, error, GPU seconds, steps."""
    import torch
    from .solver import Solver
    s = Solver(dim, degree, (elems,) * dim, velocity=(1.0, 0.0, 0.0), dtype=dtype)
    X = s.node_coords()
    U0 = inputs.random_modes(X, nk=NK, seed=seed)
    s.set_state(U0)
    dt = s.stable_dt(cfl)
    nsteps = int(math.ceil(1.0 / dt))
    dt = 1.0 / nsteps
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s.stream)
    s.step(dt, nsteps, rk)
    b.record(s.stream)
    b.synchronize()
    err = s.norms(U0)["l2"]
    out = {"dim": dim, "degree": degree, "order": degree + 1, "elems": elems, "rk": rk, "cfl": cfl,
           "dtype": dtype, "dof": s.ndof, "nsteps": nsteps, "l2_error": err,
           "gpu_seconds": a.elapsed_time(b) * 1e-3}
    s.close()
    return out


def rates(rows):
    """Observed convergence rates between consecutive refinements (error ~ DOF^-rate in 1D)."""
    out = []
    for r0, r1 in zip(rows, rows[1:]):
        if r0["l2_error"] > 0 and r1["l2_error"] > 0:
            out.append(math.log(r0["l2_error"] / r1["l2_error"]) / math.log(r1["dof"] / r0["dof"]))
    return out


def dof_for_error(rows, target):
    """DOF at which the error crosses target (log-log interpolation), or None."""
    for r0, r1 in zip(rows, rows[1:]):
        e0, e1 = r0["l2_error"], r1["l2_error"]
        if e0 >= target >= e1 > 0:
            t = (math.log(e0) - math.log(target)) / (math.log(e0) - math.log(e1))
            return math.exp(math.log(r0["dof"]) + t * (math.log(r1["dof"]) - math.log(r0["dof"])))
    return None


def study_orders(degrees=range(2, 8), cfl=0.2):
    res = {}
    for N in degrees:
        rows = [run_case(1, N, E, 6, cfl) for E in (8, 16, 32, 64, 128, 256)]
        p = N + 1
        res[N] = {"rows": rows, "rates": rates(rows), "dof_1pct": dof_for_error(rows, 1e-2),
                  "kreiss_oliger_1pct": 200.0 * (1.0 / 1e-2) ** (1.0 / p),
                  "dof_1e-4": dof_for_error(rows, 1e-4),
                  "kreiss_oliger_1e-4": 200.0 * (1.0 / 1e-4) ** (1.0 / p)}
    return res


def study_rk(degree=5, cfl=0.4):
    res = {}
    for rk in (3, 4, 6):
        rows = [run_case(1, degree, E, rk, cfl) for E in (32, 64, 128, 256, 512, 1024)]
        res[rk] = {"rows": rows, "rates": rates(rows)}
    return res


def study_time2d(degrees=range(2, 8), cfl=0.2):
    res = {}
    for N in degrees:
        res[N] = [run_case(2, N, E, 6, cfl) for E in (16, 32, 64, 128)]
    return res


def study_rk_time2d(degree=7, cfl=0.2):
    res = {}
    for rk in (3, 4, 6):
        res[rk] = [run_case(2, degree, E, rk, cfl) for E in (16, 32, 64, 128)]
    return res


STUDIES = {"orders": study_orders, "rk": study_rk, "time2d": study_time2d, "rk_time2d": study_rk_time2d}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("studies", nargs="*", default=list(STUDIES))
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    out = {name: STUDIES[name]() for name in args.studies}
    text = json.dumps(out, indent=1, default=str)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    else:
        sys.stdout.write(text + "\n")


if __name__ == "__main__":
    main()
