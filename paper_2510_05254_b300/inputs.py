"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle's tests.

This module holds no arithmetic of the DG method: only a counter-based random generator
(SplitMix64, Steele, Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
and closed-form initial conditions evaluated at coordinates that the caller supplies (node
coordinates come from whichever side -- oracle or library -- the caller trusts).

Initial conditions follow the paper's workloads:
  * ``sine``: U0 = sin(2 pi x) (1D advection, Sec. 3.1).
  * ``random_modes``: U0 = sum_{k=1}^{Nk} A_k sin(2 pi k x), A_k in [0, 1) (Eq. (initialCond)).
  * ``gaussian_noise``: 2D advection pulse exp(-r^2/0.01) at (0.5, 0.5), periodic images, plus
    seeded low-mode Fourier noise of total amplitude <= 1e-3.
  * ``euler_shear``: 2D isothermal Euler, rho = 1 + 0.1 sin(2 pi x) sin(2 pi y), velocity from a
    seeded stream function of modes |k|_inf <= 3, |u| <= 0.3 (Mach <= 0.3 at c = 1).
  * ``taylor_green``: 3D isothermal Euler, rho = 1, u = 0.1 sin cos cos, v = -0.1 cos sin cos, w = 0.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1
BASE_SEED = 20251005


class SplitMix64:
    """SplitMix64 counter-based generator; ``uniform()`` returns doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, n: int | None = None):
        if n is None:
            return (self.next_u64() >> 11) * (1.0 / (1 << 53))
        return np.array([(self.next_u64() >> 11) * (1.0 / (1 << 53)) for _ in range(n)])


def sine(X: np.ndarray) -> np.ndarray:
    """U0 = sin(2 pi x); X has shape (dim, ...). Returns shape (1, ...)."""
    return np.sin(2.0 * math.pi * X[0])[None]


def random_modes(X: np.ndarray, nk: int = 40, seed: int = BASE_SEED) -> np.ndarray:
    """U0 = sum_{k=1}^{nk} A_k sin(2 pi k x) with A_k ~ U[0,1) from SplitMix64(seed)."""
    A = SplitMix64(seed).uniform(nk)
    u = np.zeros_like(X[0])
    for k in range(1, nk + 1):
        u += A[k - 1] * np.sin(2.0 * math.pi * k * X[0])
    return u[None]


def _noise_modes(seed: int, kmax: int = 4):
    g = SplitMix64(seed)
    modes = []
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            if max(abs(kx), abs(ky)) >= 1:
                modes.append((kx, ky, g.uniform(), 2.0 * math.pi * g.uniform()))
    total = sum(m[2] for m in modes)
    return [(kx, ky, 1e-3 * a / total, ph) for kx, ky, a, ph in modes]


def gaussian_noise(X: np.ndarray, seed: int = BASE_SEED + 1, shift=(0.0, 0.0)) -> np.ndarray:
    """2D pulse exp(-r^2/0.01) at (0.5, 0.5) summed over the 3x3 periodic images, plus
    Fourier noise sum eps_k cos(2 pi k.x + phi_k) over 1 <= |k|_inf <= 4 with sum eps_k = 1e-3.
    ``shift`` evaluates U0(x - shift) (the exact solution of advection at time t is
    U0(x - a t)).  Coordinates are wrapped to [0, 1) first."""
    x = np.mod(X[0] - shift[0], 1.0)
    y = np.mod(X[1] - shift[1], 1.0)
    u = np.zeros_like(x)
    for sx in (-1.0, 0.0, 1.0):
        for sy in (-1.0, 0.0, 1.0):
            u += np.exp(-((x - 0.5 + sx) ** 2 + (y - 0.5 + sy) ** 2) / 0.01)
    for kx, ky, eps, ph in _noise_modes(seed):
        u += eps * np.cos(2.0 * math.pi * (kx * x + ky * y) + ph)
    return u[None]


def euler_shear(X: np.ndarray, seed: int = BASE_SEED + 2, umax: float = 0.3) -> np.ndarray:
    """2D isothermal Euler state (rho, rho u, rho v).  psi = sum c_k sin(2 pi k.x + phi_k) over
    1 <= |k|_inf <= 3; u = d psi/dy, v = -d psi/dx, scaled so that the bound
    sum |c_k| 2 pi |k|_2 on |u| equals umax."""
    g = SplitMix64(seed)
    modes = []
    for kx in range(-3, 4):
        for ky in range(-3, 4):
            if max(abs(kx), abs(ky)) >= 1:
                modes.append((kx, ky, g.uniform() - 0.5, 2.0 * math.pi * g.uniform()))
    bound = sum(abs(c) * 2.0 * math.pi * math.hypot(kx, ky) for kx, ky, c, _ in modes)
    s = umax / bound
    x, y = X[0], X[1]
    u = np.zeros_like(x)
    v = np.zeros_like(x)
    for kx, ky, c, ph in modes:
        cph = np.cos(2.0 * math.pi * (kx * x + ky * y) + ph)
        u += s * c * 2.0 * math.pi * ky * cph
        v -= s * c * 2.0 * math.pi * kx * cph
    rho = 1.0 + 0.1 * np.sin(2.0 * math.pi * x) * np.sin(2.0 * math.pi * y)
    return np.stack([rho, rho * u, rho * v])


def _grid_to_elements(G: np.ndarray, E: int, n: int) -> np.ndarray:
    """(E n, E n) array over (y, x) grid points -> element layout (E^2, n^2), e = ex + E ey,
    node = i + n j."""
    return G.reshape(E, n, E, n).transpose(0, 2, 1, 3).reshape(E * E, n * n)


def gaussian_noise_grid(x: np.ndarray, seed: int = BASE_SEED + 1) -> np.ndarray:
    """``gaussian_noise`` on the tensor grid whose points along each axis are the 1D coordinates
    x[ex n + i] (E elements of n nodes, the same along y), as an (E n, E n) array over (y, x).
    Both terms separate: the pulse into exp(-dx^2/0.01) exp(-dy^2/0.01) and each noise mode into
    cos a cos b - sin a sin b, so the work is one matrix product instead of ~90 transcendental
    evaluations per point (large serving grids)."""
    x = np.mod(np.asarray(x, dtype=np.float64), 1.0)
    gx = [np.exp(-((x - 0.5 + sx) ** 2) / 0.01) for sx in (-1.0, 0.0, 1.0)]
    A = [np.outer(gy, gx_) for gy in gx for gx_ in gx]  # the nine periodic images
    G = np.sum(A, axis=0)
    cols_y, cols_x = [], []
    for kx, ky, eps, ph in _noise_modes(seed):
        a = 2.0 * math.pi * kx * x + ph
        b = 2.0 * math.pi * ky * x
        cols_y += [eps * np.cos(b), -eps * np.sin(b)]
        cols_x += [np.cos(a), np.sin(a)]
    G += np.stack(cols_y, axis=1) @ np.stack(cols_x, axis=0)
    return G


def euler_shear_grid(x: np.ndarray, seed: int = BASE_SEED + 2, umax: float = 0.3) -> np.ndarray:
    """``euler_shear`` on the same tensor grid as ``gaussian_noise_grid``, as (3, E n, E n) over
    (y, x); every mode separates as there."""
    g = SplitMix64(seed)
    modes = []
    for kx in range(-3, 4):
        for ky in range(-3, 4):
            if max(abs(kx), abs(ky)) >= 1:
                modes.append((kx, ky, g.uniform() - 0.5, 2.0 * math.pi * g.uniform()))
    bound = sum(abs(c) * 2.0 * math.pi * math.hypot(kx, ky) for kx, ky, c, _ in modes)
    s = umax / bound
    x = np.asarray(x, dtype=np.float64)
    uy, vy, cx = [], [], []
    for kx, ky, c, ph in modes:
        a = 2.0 * math.pi * kx * x + ph
        b = 2.0 * math.pi * ky * x
        fu = s * c * 2.0 * math.pi * ky
        fv = -s * c * 2.0 * math.pi * kx
        uy += [fu * np.cos(b), -fu * np.sin(b)]
        vy += [fv * np.cos(b), -fv * np.sin(b)]
        cx += [np.cos(a), np.sin(a)]
    C = np.stack(cx, axis=0)
    u = np.stack(uy, axis=1) @ C
    v = np.stack(vy, axis=1) @ C
    sn = np.sin(2.0 * math.pi * x)
    rho = 1.0 + 0.1 * np.outer(sn, sn)
    return np.stack([rho, rho * u, rho * v])


def grid_state(kind: str, x: np.ndarray, E: int, n: int, seed: int) -> np.ndarray:
    """A 2D initial condition on the E x E element grid of n-node lines (1D node coordinates x of
    length E n), in the solver's element layout (nvar, E^2, n^2)."""
    G = gaussian_noise_grid(x, seed)[None] if kind == "gaussian_noise" else euler_shear_grid(x, seed)
    return np.stack([_grid_to_elements(Gv, E, n) for Gv in G])


def taylor_green(X: np.ndarray, amp: float = 0.1) -> np.ndarray:
    """3D isothermal Euler state (rho, rho u, rho v, rho w) with rho = 1 and a Taylor-Green
    velocity field of amplitude amp."""
    x, y, z = (2.0 * math.pi * X[0], 2.0 * math.pi * X[1], 2.0 * math.pi * X[2])
    rho = np.ones_like(x)
    u = amp * np.sin(x) * np.cos(y) * np.cos(z)
    v = -amp * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(x)
    return np.stack([rho, rho * u, rho * v, rho * w])


def random_state(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform random array (for operator tests on non-smooth data).  Vectorised
    SplitMix64 over a counter, so large arrays are cheap."""
    n = int(np.prod(shape))
    with np.errstate(over="ignore"):
        c = (np.arange(1, n + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
             + np.uint64(seed & _MASK))
        z = c
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return (lo + (hi - lo) * u).reshape(shape)


def serving_stream(n: int, seed: int = BASE_SEED + 5, emin: int = 16, emax: int = 512,
                   degrees=(3, 5, 7)):
    """Requests of the mixed serving workload: equation 50/50 (0 advection, 1 isothermal Euler),
    elements per axis log-uniform in [emin, emax], degree uniform in ``degrees``, dtype 50/50
    ('f64' / 'f32'), and an exponential inter-arrival draw (unit rate, scaled by the caller)."""
    g = SplitMix64(seed)
    out = []
    for i in range(n):
        eq = 0 if g.uniform() < 0.5 else 1
        E = int(round(math.exp(math.log(emin) + (math.log(emax) - math.log(emin)) * g.uniform())))
        N = degrees[min(int(g.uniform() * len(degrees)), len(degrees) - 1)]
        dtype = "f64" if g.uniform() < 0.5 else "f32"
        gap = -math.log(1.0 - g.uniform())
        out.append({"id": i, "equation": eq, "elems": E, "degree": N, "dtype": dtype, "gap": gap,
                    "seed": BASE_SEED + 1000 + i})
    return out
