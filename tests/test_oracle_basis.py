"""Pins of the oracle's LGL basis (Sec. 2.1, Eq. (lag_coefs), Eq. (lagrange_pol)) against
closed forms and identities that the mathematics fixes, independent of the oracle's code."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lgl_closed_forms.txt")


def _golden():
    rows = {}
    env = {"sqrt": math.sqrt}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        N, x, w = line.split()
        rows.setdefault(int(N), []).append((eval(x, env), eval(w, env)))
    return rows


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_lgl_closed_forms(N):
    xi, w = orc.lgl(N)
    ref = _golden()[N]
    np.testing.assert_allclose(xi, [r[0] for r in ref], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [r[1] for r in ref], rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", range(1, 16))
def test_lgl_weights_sum_and_symmetry(N):
    xi, w = orc.lgl(N)
    assert abs(w.sum() - 2.0) < 1e-14
    np.testing.assert_allclose(xi, -xi[::-1], atol=1e-15)
    np.testing.assert_allclose(w, w[::-1], atol=1e-15)
    assert np.all(np.diff(xi) > 0)


@pytest.mark.parametrize("N", range(2, 12))
def test_interior_nodes_are_roots_of_dPN(N):
    xi, _ = orc.lgl(N)
    dP = npleg.Legendre.basis(N).deriv()
    assert np.max(np.abs(dP(xi[1:-1]))) < 1e-12 * N * N
    np.testing.assert_allclose(np.sort(dP.roots().real), xi[1:-1], atol=1e-14)


@pytest.mark.parametrize("N", range(1, 12))
def test_quadrature_exact_to_degree_2N_minus_1(N):
    xi, w = orc.lgl(N)
    for m in range(0, 2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, xi ** m) - exact) < 1e-14, m
    # and not beyond: Lobatto (not Gauss) quadrature misses x^(2N) for N >= 1
    m = 2 * N
    assert abs(np.dot(w, xi ** m) - 2.0 / (m + 1)) > 1e-9


@pytest.mark.parametrize("N", range(1, 12))
def test_dmat_exact_on_polynomials_up_to_degree_N(N):
    xi, _ = orc.lgl(N)
    D = orc.dmat(N)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12)  # D 1 = 0
    for m in range(1, N + 1):
        np.testing.assert_allclose(D @ xi ** m, m * xi ** (m - 1), atol=1e-12 * N * N)


@pytest.mark.parametrize("N", range(1, 12))
def test_dmat_matches_interpolation_derivative(N):
    """D from a Legendre Vandermonde built by numpy (V_x V^{-1}), not from the oracle's formula."""
    xi, _ = orc.lgl(N)
    V = npleg.legvander(xi, N)
    Vx = np.zeros_like(V)
    for j in range(N + 1):
        Vx[:, j] = npleg.Legendre.basis(j).deriv()(xi)
    D_ref = Vx @ np.linalg.inv(V)
    np.testing.assert_allclose(orc.dmat(N), D_ref, atol=1e-12 * N * N)


@pytest.mark.parametrize("N", range(1, 12))
def test_summation_by_parts(N):
    """W D + D^T W = diag(-1, 0, ..., 0, 1): the discrete integration by parts that makes the weak
    form of Sec. 2.1 equal the strong form."""
    _, w = orc.lgl(N)
    D = orc.dmat(N)
    W = np.diag(w)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    np.testing.assert_allclose(W @ D + D.T @ W, B, atol=1e-13 * N * N)


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_lagrange_formula_of_paper_is_cardinal(N):
    """The paper's h_k (Eq. (lagrange_pol)) evaluated near the nodes: h_k(xi_l) = delta_kl
    (Eq. (ortho_at_roots)), and its derivative agrees with the oracle's D."""
    xi, _ = orc.lgl(N)
    PN = npleg.Legendre.basis(N)
    dPN = PN.deriv()

    def h(k, x):
        return (x - 1) * (x + 1) * dPN(x) / (N * (N + 1) * PN(xi[k]) * (x - xi[k]))

    D = orc.dmat(N)
    eps = 1e-6
    for k in range(N + 1):
        for l in range(N + 1):
            x = xi[l] + (eps if l < N else -eps)  # approach the node from inside [-1, 1]
            val = h(k, x)
            assert abs(val - (1.0 if k == l else 0.0)) < 1e-4
            # central difference of h_k at a point next to node l, against D[l, k]
            x0 = xi[l] + (2e-4 if l == 0 else (-2e-4 if l == N else 1e-4))
            deriv = (h(k, x0 + 1e-6) - h(k, x0 - 1e-6)) / 2e-6
            if abs(x0 - xi[k]) > 1e-3:
                assert abs(deriv - D[l, k]) < 5e-2 * (1 + abs(D[l, k]))
