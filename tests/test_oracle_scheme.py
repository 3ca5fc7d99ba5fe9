"""Pins of the oracle's NDG spatial operator and of the whole RK-NDG scheme (Sec. 2.1-2.3, 3.1)
against closed forms, invariants and brute force, none of which reuse the oracle's code."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2510_05254_b300 import inputs
from tests import bloch

ADV, EUL = orc.ADVECTION, orc.ISO_EULER


def _prob(dim, N, E, eq=ADV, flux=None, length=None, velocity=None, c=1.0):
    if flux is None:
        flux = orc.FLUX_UPWIND if eq == ADV else orc.FLUX_LLF
    E = tuple(E) if isinstance(E, (tuple, list)) else (E,) * dim
    return orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - len(E)), equation=eq, flux=flux,
                       length=tuple(length or (1.0, 1.0, 1.0)),
                       velocity=tuple(velocity or (1.0, 0.5, 0.25)), sound_speed=c)


def _quad_weights(p):
    """Per-node quadrature weights J * prod w (from numpy's LGL, not the oracle's)."""
    _, w, _ = bloch.lgl_basis(p.degree)
    n = p.n
    J = np.prod([0.5 * p.length[a] / p.elems[a] for a in range(p.dim)])
    wq = np.ones(p.npe)
    for node in range(p.npe):
        for a in range(p.dim):
            wq[node] *= w[(node // n ** a) % n]
    return J * wq  # shape (npe,)


# ------------------------------------------------------------------------------------------
# brute force: degree 1, two elements, expanded by hand from the weak form of Sec. 2.1
# ------------------------------------------------------------------------------------------

def test_bruteforce_advection_N1_two_elements():
    """N = 1: nodes -1, 1, weights 1, 1, h_0 = (1-xi)/2, h_1 = (1+xi)/2, so D = [[-1/2, 1/2],
    [-1/2, 1/2]].  With E = 2 on [0, 1] (dx = 1/2, 2/dx = 4), upwind flux, a = 1, the weak form
    (dx/2) w_l U_l' = sum_k w_k F_k D[k][l] - (Fhat_R d_l1 - Fhat_L d_l0) gives
      U_0' = 4 (U_1^left - (U_0 + U_1)/2),   U_1' = 4 (U_0 - U_1)/2.
    For a = -1 (upwind takes the right state):
      U_0' = 4 (U_1 - U_0)/2,   U_1' = 4 (U_0^right - (U_0 + U_1)/2)."""
    p, q, r, s = 1.0, 2.0, 3.0, 5.0
    U = np.array([p, q, r, s])
    P = _prob(1, 1, 2, velocity=(1.0, 0, 0))
    expect = [4 * (s - (p + q) / 2), 4 * (p - q) / 2, 4 * (q - (r + s) / 2), 4 * (r - s) / 2]
    np.testing.assert_allclose(orc.rhs(P, U).ravel(), expect, rtol=1e-15)
    P = _prob(1, 1, 2, velocity=(-1.0, 0, 0))
    expect = [4 * (q - p) / 2, 4 * (r - (p + q) / 2), 4 * (s - r) / 2, 4 * (p - (r + s) / 2)]
    np.testing.assert_allclose(orc.rhs(P, U).ravel(), expect, rtol=1e-15)
    # LLF with alpha = |a| is the same flux for advection
    P = _prob(1, 1, 2, flux=orc.FLUX_LLF, velocity=(-1.0, 0, 0))
    np.testing.assert_allclose(orc.rhs(P, U).ravel(), expect, rtol=1e-15)


def test_bruteforce_isothermal_euler_N1_two_elements():
    """1D isothermal Euler, U = (rho, m), F = (m, m^2/rho + c^2 rho) (Eq. (eulerIso2d)), local
    Lax-Friedrichs with alpha = max(|u^-|, |u^+|) + c, degree 1, E = 2, c = 0.7, hand-expanded."""
    c = 0.7
    rho = np.array([1.0, 1.5, 0.8, 1.2])  # e0: nodes 0,1; e1: nodes 0,1
    m = np.array([0.6, -0.3, 0.1, 0.5])  # |u+| > |u-| at the left face of element 0

    def F(r, mm):
        return np.array([mm, mm * mm / r + c * c * r])

    def fhat(iL, iR):
        uL, uR = np.array([rho[iL], m[iL]]), np.array([rho[iR], m[iR]])
        alpha = max(abs(m[iL] / rho[iL]), abs(m[iR] / rho[iR])) + c
        return 0.5 * (F(*uL) + F(*uR) - alpha * (uR - uL))

    out = np.zeros((2, 4))
    for e in range(2):
        i0, i1 = 2 * e, 2 * e + 1
        left_end = 2 * ((e + 1) % 2) + 1  # node 1 of the left neighbour (periodic)
        right_start = 2 * ((e + 1) % 2)   # node 0 of the right neighbour
        F0, F1 = F(rho[i0], m[i0]), F(rho[i1], m[i1])
        fL, fR = fhat(left_end, i0), fhat(i1, right_start)
        out[:, i0] = 4.0 * (-(F0 + F1) / 2 + fL)
        out[:, i1] = 4.0 * ((F0 + F1) / 2 - fR)
    P = _prob(1, 1, 2, eq=EUL, c=c)
    U = np.stack([rho, m])
    np.testing.assert_allclose(orc.rhs(P, U).reshape(2, 4), out, rtol=1e-14, atol=1e-14)


# ------------------------------------------------------------------------------------------
# invariants
# ------------------------------------------------------------------------------------------

CASES = [
    (1, 3, (5,), ADV), (2, 2, (3, 4), ADV), (3, 2, (2, 3, 2), ADV),
    (1, 4, (4,), EUL), (2, 3, (3, 2), EUL), (3, 2, (2, 2, 3), EUL),
]


def _random_state(p, seed):
    U = inputs.random_state(p.shape, seed, -1.0, 1.0)
    if p.equation == EUL:
        U[0] = 1.0 + 0.3 * U[0]       # density in [0.7, 1.3]
        U[1:] = 0.3 * U[1:]            # momentum
    return U


@pytest.mark.parametrize("dim,N,E,eq", CASES)
def test_free_stream_preservation(dim, N, E, eq):
    p = _prob(dim, N, E, eq=eq, length=(1.0, 0.7, 1.3))
    U = np.ones(p.shape)
    if eq == EUL:
        U[0] = 1.3
        for a in range(dim):
            U[1 + a] = 1.3 * (0.2 - 0.1 * a)
    R = orc.rhs(p, U)
    assert np.max(np.abs(R)) < 1e-12


@pytest.mark.parametrize("dim,N,E,eq", CASES)
def test_conservation_to_roundoff(dim, N, E, eq):
    """Telescoping numerical fluxes on a periodic grid: int R = 0 for every conserved variable,
    and the integrals are unchanged by a few RK steps."""
    p = _prob(dim, N, E, eq=eq, length=(1.0, 0.7, 1.3))
    U = _random_state(p, 11)
    wq = _quad_weights(p)
    R = orc.rhs(p, U)
    scale = np.max(np.abs(R)) * np.sum(wq) * p.nelem
    for v in range(p.nvar):
        assert abs(np.sum(R[v] * wq[None, :])) < 1e-14 * scale
    dt = 0.2 * orc.stable_dt(p, U, 0.1)
    U2 = orc.step(p, U, dt, 3, 4)
    m0 = orc.norms(p, U)["integral"]
    m1 = orc.norms(p, U2)["integral"]
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-14 * max(1.0, np.max(np.abs(m0))))


@pytest.mark.parametrize("dim,N,E", [(1, 3, (6,)), (2, 2, (3, 4)), (3, 2, (2, 3, 2))])
def test_upwind_energy_dissipation_identity(dim, N, E):
    """For upwind advection with the SBP property, d/dt (1/2)|U|_W^2 equals
    -(1/2) sum over faces of |a_n| [U]^2 integrated by the face quadrature."""
    vel = (0.8, -0.6, 0.3)
    p = _prob(dim, N, E, velocity=vel, length=(1.0, 0.7, 1.3))
    U = _random_state(p, 5)
    R = orc.rhs(p, U)
    wq = _quad_weights(p)
    rate = np.sum(wq[None, :] * U * R)
    _, w, _ = bloch.lgl_basis(N)
    n = N + 1
    Eall = list(p.elems[:dim])
    u = U[0].reshape(Eall[::-1] + [n] * dim)  # [ez][ey][ex][k][j][i]
    diss = 0.0
    for a in range(dim):
        ax_e = dim - 1 - a            # element axis of a in the reshaped array
        ax_n = dim + (dim - 1 - a)    # node axis of a
        hi = np.take(u, [N], axis=ax_n)
        lo_next = np.take(np.roll(u, -1, axis=ax_e), [0], axis=ax_n)
        jump2 = np.squeeze((lo_next - hi) ** 2, axis=ax_n)
        # face quadrature: product of LGL weights * (h_b / 2) over the other axes b
        fw = 1.0
        shape = [1] * jump2.ndim
        for b in range(dim):
            if b == a:
                continue
            fw = fw * 0.5 * p.length[b] / p.elems[b]
        wts = np.ones(jump2.shape)
        other = [b for b in range(dim) if b != a]
        node_axes = [ax for ax in range(dim, 2 * dim) if ax != ax_n]
        for b, ax in zip(sorted(other, reverse=True), node_axes):
            ax_after = ax - (1 if ax > ax_n else 0)
            sh = [1] * jump2.ndim
            sh[ax_after] = n
            wts = wts * w.reshape(sh)
        diss += abs(vel[a]) * fw * np.sum(wts * jump2)
    assert abs(rate - (-0.5 * diss)) < 1e-12 * max(1.0, diss)
    assert rate <= 0


# ------------------------------------------------------------------------------------------
# Bloch-wave closed form (block-circulant operator, one element, strong form, numpy basis)
# ------------------------------------------------------------------------------------------

def _mode_state(p, m, amp):
    """Re(exp(2 pi i m.x) amp[v]) at the oracle's nodes, and the element-0 complex vector."""
    X = orc.node_coords(p)
    phase = np.zeros(X.shape[1:])
    for a in range(p.dim):
        phase = phase + m[a] * X[a] / p.length[a]
    ph = np.exp(2j * math.pi * phase)                        # (nelem, npe)
    U = np.real(np.asarray(amp)[:, None, None] * ph[None])   # (nvar, nelem, npe)
    # element-local vector: remove the element origin phase
    origin = np.zeros(p.nelem)
    Eax = [p.elems[a] for a in range(p.dim)]
    e = np.arange(p.nelem)
    idx = [e % Eax[0]]
    if p.dim > 1:
        idx.append((e // Eax[0]) % Eax[1])
    if p.dim > 2:
        idx.append(e // (Eax[0] * Eax[1]))
    for a in range(p.dim):
        origin = origin + m[a] * idx[a] / Eax[a]
    org = np.exp(2j * math.pi * origin)                      # (nelem,)
    loc = (np.asarray(amp)[:, None] * ph[0][None] / org[0]).ravel()  # [var][node]
    return U, loc, org


def _propagate_and_compare(p, U0, loc, org, L, dt, nsteps, rk, rtol):
    Z = dt * L
    if rk in (3, 4):
        P = bloch.taylor_poly(Z, rk)  # any s-stage order-s explicit RK has R = Taylor poly
    else:
        P = bloch.expm(Z)             # RK6: compare with the exact flow (O(dt^7) per step)
    v = np.linalg.matrix_power(P, nsteps) @ loc
    ref = np.real(org[None, :, None] * v.reshape(p.nvar, 1, p.npe))
    out = orc.step(p, U0, dt, nsteps, rk)
    err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
    assert err < rtol, err


@pytest.mark.parametrize("rk", [3, 4])
@pytest.mark.parametrize("dim,N,E,m", [(1, 3, (7,), (2,)), (1, 6, (4,), (1,)),
                                       (2, 2, (3, 5), (1, 2)), (2, 4, (2, 3), (1, -1)),
                                       (3, 2, (2, 3, 2), (1, 1, -1))])
def test_bloch_wave_advection(dim, N, E, m, rk):
    vel = (0.9, -0.4, 0.35)
    L = (1.0, 0.8, 1.25)
    p = _prob(dim, N, E, velocity=vel, length=L)
    hs = [L[a] / E[a] for a in range(dim)]
    thetas = [2 * math.pi * m[a] / E[a] for a in range(dim)]
    Lop = bloch.element_operator(dim, N, [[[vel[a]]] for a in range(dim)],
                                 [abs(vel[a]) for a in range(dim)], hs, thetas)
    U0, loc, org = _mode_state(p, m, [1.0 + 0.5j])
    dt = 0.5 * orc.stable_dt(p, U0, 0.2)
    _propagate_and_compare(p, U0, loc, org, Lop, dt, 6, rk, 1e-12)


def test_bloch_wave_advection_rk6_against_exact_flow():
    p = _prob(2, 3, (3, 4), velocity=(0.7, 0.3, 0), length=(1.0, 0.9, 1.0))
    thetas = [2 * math.pi * 1 / 3, 2 * math.pi * 1 / 4]
    Lop = bloch.element_operator(2, 3, [[[0.7]], [[0.3]]], [0.7, 0.3], [1 / 3, 0.9 / 4], thetas)
    U0, loc, org = _mode_state(p, (1, 1), [0.3 - 1.0j])
    dt = orc.stable_dt(p, U0, 0.05)
    _propagate_and_compare(p, U0, loc, org, Lop, dt, 5, 6, 1e-10)


def _euler_jacobian(dim, rho, u, c, a):
    """Flux Jacobian dF_a/dU of Eq. (eulerIso2d) at (rho, rho u): derived by hand from
    F_a = (m_a, m_b m_a / rho + delta_ab c^2 rho)."""
    nv = dim + 1
    A = np.zeros((nv, nv))
    A[0, 1 + a] = 1.0
    for b in range(dim):
        A[1 + b, 0] = -u[b] * u[a] + (c * c if a == b else 0.0)
        for e in range(dim):
            A[1 + b, 1 + e] = (u[a] if b == e else 0.0) + (u[b] if a == e else 0.0)
    return A


@pytest.mark.parametrize("dim,N,E,m", [(1, 3, (4,), (1,)), (2, 3, (3, 2), (1, -1)),
                                       (3, 2, (2, 2, 3), (1, 0, 1))])
def test_bloch_wave_linearised_isothermal_euler(dim, N, E, m):
    """Small perturbation eps of a moving background (rho0 = 2, u0 = (0.3, -0.2, 0.15), c = 0.8):
    the oracle must follow the linearised discrete dynamics (LF with alpha = |u0_a| + c) to
    O(eps) relative.  Pins every flux term, its sign and the LLF alpha at first order."""
    c = 0.8
    rho0 = 2.0
    u0 = np.array([0.3, -0.2, 0.15])[:dim]
    L = (1.0, 0.8, 1.25)
    p = _prob(dim, N, E, eq=EUL, length=L, c=c)
    hs = [L[a] / E[a] for a in range(dim)]
    thetas = [2 * math.pi * m[a] / E[a] for a in range(dim)]
    As = [_euler_jacobian(dim, rho0, u0, c, a) for a in range(dim)]
    alphas = [abs(u0[a]) + c for a in range(dim)]
    Lop = bloch.element_operator(dim, N, As, alphas, hs, thetas)
    eps = 1e-7
    amp = eps * (np.array([1.0, 0.5j, -0.3, 0.2 + 0.1j])[:dim + 1])
    Up, loc, org = _mode_state(p, m, amp)
    bg = np.concatenate([[rho0], rho0 * u0])
    U0 = Up + bg[:, None, None]
    dt = 0.5 * orc.stable_dt(p, U0, 0.2)
    nsteps = 5
    P = bloch.taylor_poly(dt * Lop, 4)
    v = np.linalg.matrix_power(P, nsteps) @ loc
    ref = np.real(org[None, :, None] * v.reshape(p.nvar, 1, p.npe))
    out = orc.step(p, U0, dt, nsteps, 4) - bg[:, None, None]
    err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
    assert err < 1e-5, err


# ------------------------------------------------------------------------------------------
# the whole scheme against the exact translated solution (Sec. 3.1)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_convergence_order_exact_translation(N):
    """1D advection, U0 = sin(2 pi x), RK6 with a small step: L2 error ~ dx^(N+1)."""
    errs = []
    Es = (8, 16) if N >= 3 else (16, 32)
    for E in Es:
        p = _prob(1, N, (E,), velocity=(1.0, 0, 0))
        X = orc.node_coords(p)
        U0 = inputs.sine(X)
        T = 0.25
        dt0 = orc.stable_dt(p, U0, 0.05)
        nsteps = int(math.ceil(T / dt0))
        U = orc.step(p, U0, T / nsteps, nsteps, 6)
        exact = inputs.sine(X - T)
        errs.append(orc.norms(p, U, exact)["l2"])
    rate = math.log2(errs[0] / errs[1])
    assert rate > N + 1 - 0.4, (N, errs, rate)


def test_config1_one_revolution():
    """The 1D workload: E = 64, N = 3, sin(2 pi x), upwind, RK4 at CFL 0.1 to t = 1: the result
    is close to U0 (one revolution)."""
    p = _prob(1, 3, (64,), velocity=(1.0, 0, 0))
    X = orc.node_coords(p)
    U0 = inputs.sine(X)
    dt = orc.stable_dt(p, U0, 0.1)
    nsteps = int(math.ceil(1.0 / dt))
    U = orc.step(p, U0, 1.0 / nsteps, nsteps, 4)
    n = orc.norms(p, U, U0)
    assert n["l2"] < 1e-7 and n["linf"] < 1e-6, n


def test_time_step_rule():
    p = _prob(2, 2, (4, 5), velocity=(0.5, -1.5, 0), length=(1.0, 2.0, 1.0))
    U = np.zeros(p.shape)
    # N = 2: smallest LGL gap is 1; h_min = min(1/4, 2/5)/2 * 1; lambda = 0.5 + 1.5
    assert abs(orc.stable_dt(p, U, 0.3) - 0.3 * (0.25 / 2) / 2.0) < 1e-16
    pe = _prob(2, 1, (2, 2), eq=EUL, c=2.0)
    Ue = np.ones(pe.shape)
    Ue[1] = 0.5
    Ue[2] = -0.25
    # N = 1: gap 2, h_min = 0.5/2*2 = 0.5; lambda = 0.5 + 0.25 + 2*2
    assert abs(orc.stable_dt(pe, Ue, 1.0) - 0.5 / 4.75) < 1e-15
