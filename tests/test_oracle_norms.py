"""Pins of the oracle's norms and conserved integrals (Sec. 3.1: L2 = sqrt(int (U - U_ref)^2 dx),
evaluated by LGL quadrature on every element with the Jacobian prod_a h_a / 2).

Each check compares the oracle with something the mathematics fixes and that shares none of its
code: closed-form integrals of trigonometric products on domains of non-unit length, integrals
of global monomials (which the (N+1)-point LGL rule integrates exactly up to degree 2N - 1 on
every element, and not at degree 2N), the maximum of |U - ref| taken by numpy, and a count of
the non-finite values planted in a state.  A missing square root, a missing or wrong Jacobian, a
weight taken on the wrong axis, a wrong variable index or a reference subtracted with the wrong
sign each fail at least one of them."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2510_05254_b300 import inputs
from tests import bloch

ADV, EUL = orc.ADVECTION, orc.ISO_EULER
LENGTHS = (1.3, 0.7, 2.1)


def _prob(dim, N, E, eq=ADV, length=LENGTHS):
    E = tuple(E) if isinstance(E, (tuple, list)) else (E,) * dim
    return orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - len(E)), equation=eq,
                       flux=orc.FLUX_UPWIND if eq == ADV else orc.FLUX_LLF, length=tuple(length),
                       velocity=(1.0, 0.5, 0.25))


@pytest.mark.parametrize("dim,N,E", [(1, 5, 24), (1, 7, 12), (2, 5, (20, 18)), (2, 7, (10, 9)),
                                     (3, 5, (10, 9, 11)), (3, 7, (6, 5, 7))])
def test_l2_of_trigonometric_products_closed_form(dim, N, E):
    """U = prod_a sin(2 pi k_a x_a / L_a) with k = (1, 2, 3): int U^2 = prod_a L_a / 2 exactly, so
    L2 = sqrt(prod L_a / 2) (missing sqrt or Jacobian: off by orders of magnitude).  The quadrature
    error at these resolutions is far below the 1e-12 bound."""
    p = _prob(dim, N, E)
    X = orc.node_coords(p)
    U = np.ones((1, p.nelem, p.npe))
    for a in range(dim):
        U[0] *= np.sin(2 * np.pi * (a + 1) * X[a] / p.length[a])
    vol = np.prod(p.length[:dim])
    r = orc.norms(p, U)
    assert abs(r["l2"] - math.sqrt(vol / 2 ** dim)) < 1e-12 * math.sqrt(vol)
    # the integral of the product of sines vanishes; of 1 + U it is the volume
    assert abs(r["integral"][0]) < 1e-12 * vol
    r1 = orc.norms(p, 1.0 + U)
    assert abs(r1["integral"][0] - vol) < 1e-12 * vol
    # U - ref with ref = U / 2 halves the norm; ref = -U (wrong sign of the subtraction) would not
    r2 = orc.norms(p, U, 0.5 * U)
    assert abs(r2["l2"] - 0.5 * math.sqrt(vol / 2 ** dim)) < 1e-12 * math.sqrt(vol)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("N", [2, 3, 5])
def test_monomials_integrated_exactly_to_degree_2N_minus_1(dim, N):
    """int_0^L x^k dx = L^(k+1)/(k+1).  A product of per-axis powers with different exponents on
    different axes is integrated exactly while every exponent is <= 2N - 1 (each element's LGL
    rule is exact to that degree); exponent 2N is not (the rule is Lobatto, not more).  The
    exponents differ between axes and variables, so a weight taken on the wrong axis or an
    integral stored under the wrong variable shows."""
    p = _prob(dim, N, (3, 2, 4)[:dim], eq=EUL)
    X = orc.node_coords(p)
    nv = p.nvar
    rng = np.random.default_rng(7 + N + dim)
    U = np.zeros(p.shape)
    want = np.zeros(nv)
    for v in range(nv):
        ks = rng.integers(0, 2 * N, size=dim)  # each exponent in 0 .. 2N - 1
        ks[v % dim] = 2 * N - 1 - v % 2        # the top degree (or one below) on some axis
        term = np.ones((p.nelem, p.npe))
        exact = 1.0
        for a in range(dim):
            term *= X[a] ** ks[a]
            exact *= p.length[a] ** (ks[a] + 1) / (ks[a] + 1)
        U[v] = term + (1.0 if v == 0 else 0.0)  # density >= 1 (Euler) : integral + volume
        want[v] = exact + (np.prod(p.length[:dim]) if v == 0 else 0.0)
    r = orc.norms(p, U)
    np.testing.assert_allclose(r["integral"], want, rtol=1e-13, atol=0)
    # degree 2N along one axis: the LGL rule is no longer exact
    U2 = X[0] ** (2 * N)
    exact2 = p.length[0] ** (2 * N + 1) / (2 * N + 1) * np.prod(p.length[1:dim])
    r2 = orc.norms(_prob(dim, N, (3, 2, 4)[:dim]), U2[None])
    assert abs(r2["integral"][0] - exact2) > 1e-10 * exact2


@pytest.mark.parametrize("dim,N", [(1, 3), (2, 4), (3, 2)])
def test_l2_of_a_polynomial_is_exact(dim, N):
    """U = x^p with 2p <= 2N - 1: int U^2 = L^(2p+1)/(2p+1) times the other lengths, so the
    squared L2 norm is exact to rounding (pins the square and the square root together)."""
    p = _prob(dim, N, (4, 3, 2)[:dim])
    X = orc.node_coords(p)
    pw = N - 1 if N > 1 else 0
    a = dim - 1  # along the last axis: the weight of that axis must be the one applied
    U = (X[a] ** pw)[None]
    exact = p.length[a] ** (2 * pw + 1) / (2 * pw + 1) * np.prod([p.length[b] for b in range(dim) if b != a])
    r = orc.norms(p, U)
    assert abs(r["l2"] ** 2 - exact) < 1e-13 * exact
    assert abs(r["l2"] - math.sqrt(exact)) < 1e-13 * math.sqrt(exact)


@pytest.mark.parametrize("dim,N,E,eq", [(1, 3, (5,), ADV), (2, 4, (3, 2), EUL), (3, 2, (2, 3, 2), EUL),
                                        (2, 7, (2, 3), ADV)])
def test_norms_match_an_independent_quadrature_on_random_states(dim, N, E, eq):
    """L2 / Linf / integrals against numpy: weights from the moment equations (tests/bloch.py, not
    the oracle's Newton iteration) times the Jacobian, with and without a reference state."""
    p = _prob(dim, N, E, eq=eq)
    _, w, _ = bloch.lgl_basis(N)
    n = N + 1
    J = np.prod([0.5 * p.length[a] / p.elems[a] for a in range(dim)])
    idx = np.arange(p.npe)
    wq = np.full(p.npe, J)
    for a in range(dim):
        wq = wq * w[(idx // n ** a) % n]
    U = inputs.random_state(p.shape, 31, -1.0, 1.0)
    ref = inputs.random_state(p.shape, 32, -1.0, 1.0)
    for r_ in (None, ref):
        d = U - (r_ if r_ is not None else 0.0)
        got = orc.norms(p, U, r_)
        l2 = math.sqrt(float(np.sum(wq[None, None, :] * d * d)))
        assert abs(got["l2"] - l2) < 1e-14 * l2
        assert got["linf"] == np.abs(d).max()
        np.testing.assert_allclose(got["integral"], np.sum(wq[None, None, :] * U, axis=(1, 2)),
                                   rtol=1e-13, atol=1e-15)
        assert got["nonfinite"] == 0


def test_linf_and_nonfinite_count():
    """Linf is the largest |U - ref| wherever it sits (the last variable's last node here); NaN
    and infinities are counted one by one."""
    p = _prob(2, 3, (3, 2), eq=EUL)
    U = inputs.random_state(p.shape, 5, -0.5, 0.5)
    U[-1, -1, -1] = -7.25
    got = orc.norms(p, U)
    assert got["linf"] == 7.25 and got["nonfinite"] == 0
    ref = np.zeros(p.shape)
    ref[-1, -1, -1] = -7.0
    assert orc.norms(p, U, ref)["linf"] == np.abs(U - ref).max()
    U[0, 0, 0] = np.nan
    U[1, 2, 3] = np.inf
    U[2, 5, 15] = -np.inf
    assert orc.norms(p, U)["nonfinite"] == 3
