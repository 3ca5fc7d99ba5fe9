"""The oracle's exact-mass variant (the paper lumps the mass matrix, Eq. (lag_coefs); the NDG
textbook it cites integrates it exactly: the option mass = MASS_EXACT), pinned against closed
forms and an independent strong-form operator, none of which reuse the oracle's code."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from tests import bloch

ADV, EUL = orc.ADVECTION, orc.ISO_EULER


def _prob(dim, N, E, eq=ADV, length=(1.0, 0.8, 1.25), velocity=(0.9, -0.4, 0.35), c=1.0):
    flux = orc.FLUX_UPWIND if eq == ADV else orc.FLUX_LLF
    E = tuple(E)
    return orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - len(E)), equation=eq, flux=flux,
                       length=length, velocity=velocity, sound_speed=c, mass=orc.MASS_EXACT)


@pytest.mark.parametrize("N", range(1, 8))
def test_exact_mass_matrix(N):
    """p^T M q = int_{-1}^{1} p q for all monomials p, q of degree <= N (closed form
    2/(a+b+1) or 0); M symmetric positive definite; M 1 = w (int h_k = w_k, LGL being exact to
    degree 2N-1); the lumped option is diag(w)."""
    M = orc.mass(N, exact=True)
    xi, w = orc.lgl(N)
    for a in range(N + 1):
        for b in range(N + 1):
            exact = 0.0 if (a + b) % 2 else 2.0 / (a + b + 1)
            assert abs(xi ** a @ M @ xi ** b - exact) < 1e-14
    assert np.abs(M - M.T).max() < 1e-15
    assert np.linalg.eigvalsh(M).min() > 0
    np.testing.assert_allclose(M.sum(axis=1), w, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(orc.mass(N, exact=False), np.diag(w))
    # a degree-2N product is integrated exactly, which the lumped quadrature misses
    assert abs(xi ** N @ M @ xi ** N - 2.0 / (2 * N + 1)) < 1e-14
    assert abs(xi ** N @ np.diag(w) @ xi ** N - 2.0 / (2 * N + 1)) > 1e-5


def _random_bloch_state(p, m, seed):
    """U_e = Re(exp(i theta . e) loc) with an arbitrary (discontinuous) complex element vector loc:
    a Bloch mode of the block-circulant operator whatever loc is."""
    g = np.random.default_rng(seed)
    loc = g.standard_normal(p.nvar * p.npe) + 1j * g.standard_normal(p.nvar * p.npe)
    Eax = [p.elems[a] for a in range(3)]
    e = np.arange(p.nelem)
    idx = [e % Eax[0], (e // Eax[0]) % Eax[1], e // (Eax[0] * Eax[1])]
    phase = sum(m[a] * idx[a] / Eax[a] for a in range(p.dim))
    org = np.exp(2j * math.pi * phase)
    U = np.real(org[None, :, None] * loc.reshape(p.nvar, 1, p.npe))
    return U, loc, org


@pytest.mark.parametrize("dim,N,E,m", [(1, 3, (7,), (2,)), (1, 6, (4,), (1,)), (2, 2, (3, 5), (1, 2)),
                                       (2, 5, (2, 3), (1, -1)), (3, 2, (2, 3, 2), (1, 1, -1))])
def test_bloch_wave_exact_mass_advection(dim, N, E, m):
    """Six RK4 steps from a discontinuous Bloch state equal R(dt L_theta)^6 applied to it, with
    L_theta the strong-form operator lifted by M^-1 e_0 / M^-1 e_N (numpy's orthonormal Legendre
    basis); the lumped operator differs at O(1) on such a state."""
    vel = (0.9, -0.4, 0.35)
    L = (1.0, 0.8, 1.25)
    p = _prob(dim, N, E, velocity=vel, length=L)
    hs = [L[a] / E[a] for a in range(dim)]
    thetas = [2 * math.pi * m[a] / E[a] for a in range(dim)]
    As = [[[vel[a]]] for a in range(dim)]
    alphas = [abs(vel[a]) for a in range(dim)]
    Lop = bloch.element_operator(dim, N, As, alphas, hs, thetas, mass="exact")
    U0, loc, org = _random_bloch_state(p, m, 5)
    dt = 0.1 * min(hs) / sum(abs(v) for v in vel[:dim]) / (N + 1) ** 2
    P = np.linalg.matrix_power(bloch.taylor_poly(dt * Lop, 4), 6)
    ref = np.real(org[None, :, None] * (P @ loc).reshape(p.nvar, 1, p.npe))
    out = orc.step(p, U0, dt, 6, 4)
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < 1e-12
    lumped = bloch.element_operator(dim, N, As, alphas, hs, thetas, mass="lumped")
    refl = np.real(org[None, :, None] * (np.linalg.matrix_power(bloch.taylor_poly(dt * lumped, 4), 6) @ loc)
                   .reshape(p.nvar, 1, p.npe))
    assert np.max(np.abs(out - refl)) / np.max(np.abs(ref)) > 1e-4


def test_bloch_wave_exact_mass_linearised_euler():
    """Isothermal Euler around a moving background: first-order agreement with the exact-mass
    strong-form operator of the flux Jacobians (LLF alpha = |u0_a| + c)."""
    dim, N, E, m = 2, 3, (3, 2), (1, -1)
    c, rho0, u0 = 0.8, 2.0, np.array([0.3, -0.2])
    L = (1.0, 0.8, 1.25)
    p = _prob(dim, N, E, eq=EUL, length=L, c=c)
    hs = [L[a] / E[a] for a in range(dim)]
    thetas = [2 * math.pi * m[a] / E[a] for a in range(dim)]
    As = []
    for a in range(dim):
        A = np.zeros((3, 3))
        A[0, 1 + a] = 1.0
        for b in range(dim):
            A[1 + b, 0] = -u0[b] * u0[a] + (c * c if a == b else 0.0)
            for e in range(dim):
                A[1 + b, 1 + e] = (u0[a] if b == e else 0.0) + (u0[b] if a == e else 0.0)
        As.append(A)
    Lop = bloch.element_operator(dim, N, As, [abs(u0[a]) + c for a in range(dim)], hs, thetas, mass="exact")
    Up, loc, org = _random_bloch_state(p, m, 9)
    eps = 1e-7
    bg = np.concatenate([[rho0], rho0 * u0])
    U0 = eps * Up + bg[:, None, None]
    dt = 0.02 * min(hs)
    P = np.linalg.matrix_power(bloch.taylor_poly(dt * Lop, 4), 4)
    ref = np.real(org[None, :, None] * (P @ loc).reshape(p.nvar, 1, p.npe))
    out = (orc.step(p, U0, dt, 4, 4) - bg[:, None, None]) / eps
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < 1e-5


@pytest.mark.parametrize("dim,N,E,eq", [(1, 4, (6,), EUL), (2, 3, (3, 4), ADV), (2, 5, (3, 2), EUL),
                                        (3, 2, (2, 3, 2), EUL)])
def test_exact_mass_free_stream_and_conservation(dim, N, E, eq):
    """A uniform state is steady, and with a discontinuous state the integrals (LGL quadrature =
    1^T M U, since M 1 = w) are unchanged by RK steps up to round-off."""
    p = _prob(dim, N, E, eq=eq)
    U = np.ones(p.shape)
    if eq == EUL:
        U[0] = 1.4
        for a in range(dim):
            U[1 + a] = 1.4 * (0.25 - 0.1 * a)
    assert np.max(np.abs(orc.rhs(p, U))) < 1e-12
    g = np.random.default_rng(4)
    U = U + 0.05 * g.standard_normal(p.shape)
    dt = 0.1 * orc.stable_dt(p, U, 0.1)
    m0 = orc.norms(p, U)["integral"]
    m1 = orc.norms(p, orc.step(p, U, dt, 3, 4))["integral"]
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-14 * max(1.0, np.max(np.abs(m0))))


def test_exact_mass_convergence_order():
    """1D advection of sin(2 pi x) for a short time with RK6: error ~ dx^(N+1) (N = 3)."""
    N, errs = 3, []
    for E in (8, 16):
        p = _prob(1, N, (E,), velocity=(1.0, 0, 0), length=(1.0, 1.0, 1.0))
        X = orc.node_coords(p)
        U0 = np.sin(2 * math.pi * X[0])[None]
        T = 0.25
        dt0 = 0.05 / E / (N + 1)
        nsteps = int(math.ceil(T / dt0))
        U = orc.step(p, U0, T / nsteps, nsteps, 6)
        exact = np.sin(2 * math.pi * (X[0] - T))[None]
        errs.append(orc.norms(p, U, exact)["l2"])
    rate = math.log(errs[0] / errs[1]) / math.log(2.0)
    assert rate > N + 1 - 0.3, (errs, rate)
