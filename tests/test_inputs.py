"""The separable grid forms of the 2D initial conditions (used for large serving grids) equal
the pointwise forms on the same tensor grid, to rounding."""
import math

import numpy as np
import pytest

from paper_2510_05254_b300 import inputs


def _grid(E, n):
    xi = np.cos(np.pi * np.arange(n)[::-1] / (n - 1))  # any increasing nodes on [-1, 1]
    x = (np.arange(E)[:, None] / E + 0.5 / E * (xi[None, :] + 1.0)).reshape(-1)
    X = np.empty((2, E, E, n, n))
    X[0] = x.reshape(E, n)[None, :, None, :]
    X[1] = x.reshape(E, n)[:, None, :, None]
    return x, X.reshape(2, E * E, n * n)


@pytest.mark.parametrize("E,n,seed", [(5, 4, 7), (3, 8, 11), (16, 6, 123)])
def test_grid_forms_equal_pointwise(E, n, seed):
    x, X = _grid(E, n)
    a = inputs.gaussian_noise(X, seed=seed)
    b = inputs.grid_state("gaussian_noise", x, E, n, seed)
    assert b.shape == a.shape and np.abs(a - b).max() < 1e-13
    a = inputs.euler_shear(X, seed=seed)
    b = inputs.grid_state("euler_shear", x, E, n, seed)
    assert b.shape == a.shape and np.abs(a - b).max() < 1e-13
    # the element layout: element ex + E ey, node i + n j
    assert math.isclose(b[0, 1 + E * 2, 3 + n * 1], a[0, 1 + E * 2, 3 + n * 1], rel_tol=1e-13)
