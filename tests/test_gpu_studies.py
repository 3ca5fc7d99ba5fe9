"""The convergence study of Sec. 3.1 on the GPU path: observed order N+1 for 1D advection of the
random-mode profile (Eq. (initialCond)) over one revolution, the GPU errors equal to the oracle's
for the same runs, and the RK order capping the rate (Sec. 3.1, RK-order study)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2510_05254_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05254_b300 import studies  # noqa: E402


@pytest.mark.parametrize("N", [4, 5, 6])
def test_gpu_convergence_order(N):
    # Nk = 40 modes: the asymptotic rate needs a few elements per shortest wavelength (1/40)
    rows = [studies.run_case(1, N, E, 6, 0.1) for E in (64, 128, 256)]
    r = studies.rates(rows)
    assert r[-1] > N + 1 - 0.5, (N, [x["l2_error"] for x in rows], r)


def test_gpu_errors_equal_oracle_errors():
    row = studies.run_case(1, 3, 32, 4, 0.2)
    p = orc.Problem(dim=1, degree=3, elems=(32, 1, 1), equation=0, flux=0, velocity=(1.0, 0, 0))
    X = orc.node_coords(p)
    U0 = inputs.random_modes(X, nk=studies.NK)
    U = orc.step(p, U0, 1.0 / row["nsteps"], row["nsteps"], 4)
    err = orc.norms(p, U, U0)["l2"]
    assert abs(row["l2_error"] - err) < 1e-10 * max(err, 1e-300) + 1e-14


def test_rk_order_caps_the_rate():
    """Degree 5 at a large CFL: RK3's third-order time error dominates once the grid is fine,
    RK6 keeps converging faster."""
    r3 = [studies.run_case(1, 5, E, 3, 0.4) for E in (64, 128, 256)]
    r6 = [studies.run_case(1, 5, E, 6, 0.4) for E in (64, 128, 256)]
    rate3 = studies.rates(r3)[-1]
    rate6 = studies.rates(r6)[-1]
    assert 2.5 < rate3 < 3.6, rate3
    assert rate6 > rate3 + 1.0, (rate3, rate6)
