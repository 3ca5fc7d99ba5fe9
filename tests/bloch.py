"""Independent closed form for the NDG semi-discretisation of a LINEAR hyperbolic system
U_t + sum_a A_a dU/dx_a = 0 with the Lax-Friedrichs flux of fixed alpha_a (Eq. (LF)), used to pin
the oracle.

For a single Fourier mode exp(2 pi i m.x) the periodic element grid makes the semi-discrete
operator block-circulant: each element sees its neighbours multiplied by exp(+-i theta_a),
theta_a = 2 pi m_a dx_a.  The whole scheme then reduces to one (nvar n^d) x (nvar n^d) complex
matrix L_theta per element, assembled here in the STRONG form
   dU/dt = sum_a (2/dx_a) [ -(D (x) A_a) U + lift of (F - Fhat) at the two end nodes ],
with the LGL basis built from numpy's Legendre module and a moment solve for the weights, so that
nothing is shared with the oracle (which uses the weak form, its own Newton iteration and the
closed-form D).  The fully discrete solution after n steps of an explicit RK method is
R(dt L_theta)^n applied to the initial element vector, R the stability polynomial.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg


def lgl_basis(N: int):
    """Nodes (roots of P_N' plus the ends), weights from the moment equations, and D = V_x V^-1."""
    inner = np.sort(npleg.Legendre.basis(N).deriv().roots().real)
    x = np.concatenate([[-1.0], inner, [1.0]])
    M = np.vander(x, N + 1, increasing=True).T  # M[m, k] = x_k^m
    moments = np.array([0.0 if m % 2 else 2.0 / (m + 1) for m in range(N + 1)])
    w = np.linalg.solve(M, moments)
    V = npleg.legvander(x, N)
    Vx = np.zeros_like(V)
    for j in range(N + 1):
        Vx[:, j] = npleg.Legendre.basis(j).deriv()(x)
    D = Vx @ np.linalg.inv(V)
    return x, w, D


def lift_vectors(N, mass="lumped"):
    """M^-1 e_0 and M^-1 e_N: the lift of a face term onto the line's nodes.  Lumped mass: the
    end-node unit vectors over the LGL weights.  Exact mass: M^-1 = V V^T with V the orthonormal
    Legendre Vandermonde at the nodes (M = (V V^T)^-1 for an orthonormal modal basis)."""
    x, w, _ = lgl_basis(N)
    n = N + 1
    if mass == "lumped":
        l0 = np.zeros(n); l0[0] = 1.0 / w[0]
        lN = np.zeros(n); lN[N] = 1.0 / w[N]
        return l0, lN
    V = npleg.legvander(x, N) * np.sqrt((2.0 * np.arange(n) + 1.0) / 2.0)
    Minv = V @ V.T
    return Minv[:, 0], Minv[:, N]


def line_operator(N, A, alpha, h, theta, mass="lumped"):
    """(n*nvar) x (n*nvar) operator of one 1D line, ordering [node][var].  With the exact mass
    matrix the strong form keeps -D F (W D F = M D F: the LGL quadrature of h_l times a degree
    N-1 polynomial is exact) and lifts the face terms by M^-1 e_0, M^-1 e_N instead."""
    x, w, D = lgl_basis(N)
    n = N + 1
    A = np.atleast_2d(np.asarray(A, dtype=complex))
    nv = A.shape[0]
    I = np.eye(nv)
    L = -np.kron(D, A).astype(complex)
    eN = np.zeros(n); eN[N] = 1.0
    e0 = np.zeros(n); e0[0] = 1.0
    l0, lN = lift_vectors(N, mass)
    ph = np.exp(1j * theta)
    # right face: M^-1 e_N (F_N - Fhat_R) = M^-1 e_N 1/2 (A - alpha)(u_N - e^{i theta} u_0)
    L += np.kron(np.outer(lN, eN - ph * e0), 0.5 * (A - alpha * I))
    # left face: M^-1 e_0 (Fhat_L - F_0) = M^-1 e_0 1/2 (A + alpha)(e^{-i theta} u_N - u_0)
    L += np.kron(np.outer(l0, np.conj(ph) * eN - e0), 0.5 * (A + alpha * I))
    return (2.0 / h) * L


def element_operator(dim, N, As, alphas, hs, thetas, mass="lumped"):
    """Full element operator with ordering [var][node], node = i + n j + n^2 k (i fastest)."""
    n = N + 1
    nv = np.atleast_2d(As[0]).shape[0]
    npe = n ** dim
    total = np.zeros((nv * npe, nv * npe), dtype=complex)
    for a in range(dim):
        La = line_operator(N, As[a], alphas[a], hs[a], thetas[a], mass)  # [node_a][var] ordering
        La4 = La.reshape(n, nv, n, nv)  # (l, v, k, u)
        # embed: node multi-index (i0, i1, i2), axis a varies, others identity
        for base in range(npe):
            idx = [(base // n ** b) % n for b in range(dim)]
            if idx[a] != 0:
                continue
            nodes = [base + l * n ** a for l in range(n)]
            for l in range(n):
                for v in range(nv):
                    row = v * npe + nodes[l]
                    for k in range(n):
                        for u in range(nv):
                            total[row, u * npe + nodes[k]] += La4[l, v, k, u]
    return total


def taylor_poly(z_matrix, order):
    """sum_{j<=order} Z^j / j!"""
    Z = z_matrix
    out = np.eye(Z.shape[0], dtype=complex)
    term = np.eye(Z.shape[0], dtype=complex)
    for j in range(1, order + 1):
        term = term @ Z / j
        out = out + term
    return out


def expm(Z):
    """Matrix exponential by scaling and squaring of a long Taylor series."""
    nrm = np.linalg.norm(Z, 1)
    s = max(0, int(math.ceil(math.log2(max(nrm, 1e-300)))) + 1)
    Zs = Z / (2 ** s)
    E = taylor_poly(Zs, 30)
    for _ in range(s):
        E = E @ E
    return E
