"""ORACLE binding (test infrastructure only).

ctypes wrapper around ``ndg_oracle.c``: the plain single-threaded FP64 CPU implementation of the
nodal DG + Runge-Kutta method of arXiv:2510.05254, Sec. 2.  Only the tests, the smoke check and
the CPU-baseline leg of the benchmark use it; it imports nothing from the CUDA package, and the
CUDA package never imports it.

The shared library is built on first use with gcc (``-O2 -ffp-contract=off``), next to the source;
a second build of the same source with ``-O3 -march=native`` (per host CPU, under ``_build/``)
serves the timed CPU baseline, alone or split over the host's cores (``step_threads``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ndg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ADVECTION, ISO_EULER = 0, 1
FLUX_UPWIND, FLUX_LLF = 0, 1
MASS_LUMPED, MASS_EXACT = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc if the library is missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-pthread", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


def _host_tag() -> str:
    """A tag of this host's CPU (model and feature flags): a -march=native build is only valid on
    the CPU it was compiled for."""
    import hashlib
    import platform
    try:
        with open("/proc/cpuinfo") as f:
            info = [l for l in f if l.startswith(("model name", "flags", "Features"))][:2]
    except OSError:
        info = [platform.processor()]
    return hashlib.sha1("".join(info).encode()).hexdigest()[:12]


def build_timing(force: bool = False) -> str:
    """The same source for timing on this host: -O3 -march=native, still -ffp-contract=off (no
    contraction; without -ffast-math the compiler may not reorder the sums either, so results are
    bitwise those of the checking build -- tested).  Built per CPU under oracle/_build/."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, f"liboracle_native_{_host_tag()}.so")
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-march=native", "-std=c99", "-ffp-contract=off", "-pthread", "-fPIC",
                        "-shared", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, lib)
    return lib


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("degree", ctypes.c_int),
        ("elems", ctypes.c_int * 3),
        ("equation", ctypes.c_int),
        ("flux", ctypes.c_int),
        ("length", ctypes.c_double * 3),
        ("velocity", ctypes.c_double * 3),
        ("sound_speed", ctypes.c_double),
        ("mass", ctypes.c_int),
    ]


@dataclass
class Problem:
    """A uniform periodic Cartesian problem: dim, degree N, elements per axis, equation, flux."""

    dim: int
    degree: int
    elems: tuple
    equation: int = ADVECTION
    flux: int = FLUX_UPWIND
    length: tuple = (1.0, 1.0, 1.0)
    velocity: tuple = (1.0, 0.0, 0.0)
    sound_speed: float = 1.0
    mass: int = MASS_LUMPED  # the paper's lumped mass, or the exact mass matrix (reading 1)

    @property
    def nvar(self) -> int:
        return 1 if self.equation == ADVECTION else self.dim + 1

    @property
    def n(self) -> int:
        return self.degree + 1

    @property
    def nelem(self) -> int:
        return int(np.prod([self.elems[a] for a in range(self.dim)]))

    @property
    def npe(self) -> int:
        return self.n ** self.dim

    @property
    def ndof(self) -> int:
        return self.nvar * self.nelem * self.npe

    @property
    def shape(self) -> tuple:
        return (self.nvar, self.nelem, self.npe)

    def _c(self) -> _Problem:
        e = list(self.elems) + [1] * (3 - len(self.elems))
        L = list(self.length) + [1.0] * (3 - len(self.length))
        a = list(self.velocity) + [0.0] * (3 - len(self.velocity))
        return _Problem(self.dim, self.degree, (ctypes.c_int * 3)(*e[:3]), self.equation, self.flux,
                        (ctypes.c_double * 3)(*L[:3]), (ctypes.c_double * 3)(*a[:3]), self.sound_speed,
                        self.mass)


def _declare(lib):
    P = ctypes.POINTER(_Problem)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_lgl.argtypes = [ctypes.c_int, dp, dp]
    lib.orc_dmat.argtypes = [ctypes.c_int, dp, dp]
    lib.orc_mass.argtypes = [ctypes.c_int, ctypes.c_int, dp]
    lib.orc_rhs.argtypes = [P, dp, dp]
    lib.orc_step.argtypes = [P, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    lib.orc_step_threads.argtypes = [P, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_norms.argtypes = [P, dp, dp, dp]
    lib.orc_stable_dt.argtypes = [P, dp, ctypes.c_double]
    lib.orc_stable_dt.restype = ctypes.c_double
    lib.orc_node_coords.argtypes = [P, dp]
    lib.orc_ndof.argtypes = [P]
    lib.orc_ndof.restype = ctypes.c_int64
    lib.orc_rk_ode.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int, dp]
    return lib


_timing_lib = None


def _load_timing():
    global _timing_lib
    with _lock:
        if _timing_lib is None:
            _timing_lib = _declare(ctypes.CDLL(build_timing()))
    return _timing_lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def lgl(N: int):
    """LGL nodes and weights of degree N (ascending)."""
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if _load().orc_lgl(N, _ptr(xi), _ptr(w)) != 0:
        raise ValueError("bad degree")
    return xi, w


def dmat(N: int) -> np.ndarray:
    """D[k, l] = h_l'(xi_k) on the LGL nodes."""
    xi, _ = lgl(N)
    D = np.zeros((N + 1) * (N + 1))
    _load().orc_dmat(N, _ptr(xi), _ptr(D))
    return D.reshape(N + 1, N + 1)


def mass(N: int, exact: bool = True) -> np.ndarray:
    """Mass matrix of the Lagrange basis on the LGL nodes: exact (Gauss quadrature) or lumped."""
    M = np.zeros((N + 1) * (N + 1))
    if _load().orc_mass(N, int(bool(exact)), _ptr(M)) != 0:
        raise ValueError("bad degree")
    return M.reshape(N + 1, N + 1)


def node_coords(p: Problem) -> np.ndarray:
    """Node coordinates, shape (dim, nelem, npe)."""
    X = np.zeros((p.dim, p.nelem, p.npe))
    c = p._c()
    if _load().orc_node_coords(ctypes.byref(c), _ptr(X)) != 0:
        raise ValueError("bad problem")
    return X


def rhs(p: Problem, U) -> np.ndarray:
    """The semi-discrete right-hand side L(U), same layout as U."""
    U = _f64(U).reshape(p.shape)
    R = np.zeros_like(U)
    c = p._c()
    if _load().orc_rhs(ctypes.byref(c), _ptr(U), _ptr(R)) != 0:
        raise ValueError("bad problem")
    return R


def step(p: Problem, U, dt: float, nsteps: int, rk: int = 4) -> np.ndarray:
    """nsteps Runge-Kutta steps (rk in {3, 4, 6}); returns a new array."""
    U = _f64(U).reshape(p.shape).copy()
    c = p._c()
    rc = _load().orc_step(ctypes.byref(c), _ptr(U), float(dt), int(nsteps), int(rk))
    if rc != 0:
        raise ValueError(f"orc_step failed ({rc})")
    return U


def step_threads(p: Problem, U, dt: float, nsteps: int, rk: int = 4, threads: int = 0,
                 native: bool = False) -> np.ndarray:
    """The same steps split over `threads` threads by element ranges (0: every core of the host);
    bitwise equal to step().  For timing the CPU on many cores -- the checker is step().  native:
    use the -O3 -march=native build of the same source (build_timing)."""
    U = _f64(U).reshape(p.shape).copy()
    c = p._c()
    lib = _load_timing() if native else _load()
    n = threads or (os.cpu_count() or 1)
    rc = lib.orc_step_threads(ctypes.byref(c), _ptr(U), float(dt), int(nsteps), int(rk), int(n))
    if rc != 0:
        raise ValueError(f"orc_step_threads failed ({rc})")
    return U


def step_native(p: Problem, U, dt: float, nsteps: int, rk: int = 4) -> np.ndarray:
    """step() from the -O3 -march=native build (timing on this host)."""
    U = _f64(U).reshape(p.shape).copy()
    c = p._c()
    rc = _load_timing().orc_step(ctypes.byref(c), _ptr(U), float(dt), int(nsteps), int(rk))
    if rc != 0:
        raise ValueError(f"orc_step failed ({rc})")
    return U


def norms(p: Problem, U, ref=None) -> dict:
    """L2 / Linf of U - ref (ref None: of U), per-variable integrals, non-finite count."""
    U = _f64(U).reshape(p.shape)
    out = np.zeros(7)
    c = p._c()
    refp = None
    if ref is not None:
        ref = _f64(ref).reshape(p.shape)
        refp = _ptr(ref)
    _load().orc_norms(ctypes.byref(c), _ptr(U), refp, _ptr(out))
    return {"l2": out[0], "linf": out[1], "integral": out[2:2 + p.nvar].copy(), "nonfinite": int(out[6])}


def stable_dt(p: Problem, U, cfl: float) -> float:
    U = _f64(U).reshape(p.shape)
    c = p._c()
    dt = _load().orc_stable_dt(ctypes.byref(c), _ptr(U), float(cfl))
    if not dt > 0:
        raise ValueError("no stable dt")
    return dt


def rk_ode(rk: int, which: int, lam: float, y0: float, dt: float, nsteps: int) -> float:
    """Run the oracle's Runge-Kutta code on y' = lam*y (which=0) or y' = -y^2 (which=1)."""
    y = np.zeros(1)
    if _load().orc_rk_ode(rk, which, lam, y0, dt, nsteps, _ptr(y)) != 0:
        raise ValueError("bad rk")
    return float(y[0])
