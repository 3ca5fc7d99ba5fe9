"""Pins of the oracle's Runge-Kutta code (Sec. 2.3, Eq. (RK3), (RK4), (RK6)) against facts that
any method of the stated order must satisfy, independent of the printed tableaus."""
import math

import numpy as np
import pytest

from oracle import oracle as orc

STAGES = {3: 3, 4: 4, 6: 7}


def _stability_coefficients(rk):
    """Fit R(z) = y1 / y0 for y' = z y, dt = 1 (a polynomial of degree = number of stages)."""
    s = STAGES[rk]
    zs = np.linspace(-0.5, 0.5, s + 1)
    R = np.array([orc.rk_ode(rk, 0, z, 1.0, 1.0, 1) for z in zs])
    V = np.vander(zs, s + 1, increasing=True)
    return np.linalg.solve(V, R)


@pytest.mark.parametrize("rk", [3, 4, 6])
def test_stability_polynomial_is_truncated_exponential(rk):
    c = _stability_coefficients(rk)
    order = {3: 3, 4: 4, 6: 6}[rk]
    for j in range(order + 1):
        assert abs(c[j] - 1.0 / math.factorial(j)) < 1e-9, (rk, j, c[j])
    if rk in (3, 4):  # s stages, order s: R is exactly the Taylor polynomial
        assert len(c) == order + 1
    else:  # seven stages, order six: the z^7 term is not 1/7!
        assert abs(c[7] - 1.0 / math.factorial(7)) > 1e-6


@pytest.mark.parametrize("rk,order", [(3, 3), (4, 4), (6, 6)])
def test_nonlinear_convergence_order(rk, order):
    """y' = -y^2, y(0) = 1, exact y(1) = 1/2: global error ~ dt^order."""
    errs = []
    for nsteps in (8, 16, 32):
        y = orc.rk_ode(rk, 1, 0.0, 1.0, 1.0 / nsteps, nsteps)
        errs.append(abs(y - 0.5))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(rates[-1] - order) < 0.35 and rates[0] > order - 0.5, (rk, errs, rates)


def test_rk_rejects_unknown_scheme():
    with pytest.raises(ValueError):
        orc.rk_ode(5, 0, -1.0, 1.0, 0.1, 1)
