"""Degenerate grids and size limits through the C ABI.

One element along an axis makes an element its own periodic neighbour on both faces along it;
two elements make the low and the high neighbour the same element.  Every precision, both
equations, both thread mappings and the split stage must still match the FP64 oracle (FP64 and
the float-float contraction within 1e-12 per step, FP32 within its tolerance), including the
classes with bulk-copied tiles (FP32 degree 5 in 2D/3D, degree 7 in 3D).  A grid of 2^31 or more
elements is refused before any device memory is taken."""
import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05254_b300 import native as nat  # noqa: E402
from paper_2510_05254_b300.solver import Solver  # noqa: E402
from tests.test_gpu_parity import F32_TOL, F64_TOL, initial, rel_l2  # noqa: E402

GRIDS = [(1, 4, (1,)), (1, 7, (2,)), (2, 3, (1, 1)), (2, 5, (1, 3)), (2, 7, (2, 1)), (3, 2, (1, 1, 1)),
         (3, 5, (1, 2, 3)), (3, 5, (2, 2, 1)), (3, 7, (1, 1, 2)), (3, 3, (2, 1, 2))]


@pytest.mark.parametrize("eq", [0, 1])
@pytest.mark.parametrize("dim,N,E", GRIDS)
def test_one_or_two_elements_along_an_axis(dim, N, E, eq):
    flux = 0 if eq == 0 else 1
    kw = dict(equation=eq, flux=flux, length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3))
    p = orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - dim), **kw)
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    for dtype, tol in (("f64", F64_TOL), ("f64ff", F64_TOL), ("f32", 2 * F32_TOL)):
        U0 = U.astype(np.float32).astype(np.float64) if dtype == "f32" else U
        ref = orc.step(p, U0, dt, 2, 4)
        outs = []
        for kernel in (nat.NDG_KERNEL_LINE, nat.NDG_KERNEL_LINE_VAR):
            s = Solver(dim, N, E, dtype=dtype, kernel=kernel, **kw)
            s.set_state(U0)
            s.step(dt, 2, 4)
            got = s.get_state()
            assert rel_l2(got, ref) < tol, (dtype, kernel, rel_l2(got, ref))
            outs.append(got)
            if dtype != "f64ff":
                s.set_state(U0)
                nat.ndg_step_split(s.ctx, dt, 2, 4)
                assert np.array_equal(s.get_state(), got), (dtype, kernel)
            s.close()
        assert np.array_equal(outs[0], outs[1]), dtype


def test_grid_of_two_to_the_31_elements_is_refused():
    cfg = nat.ndg_config_init()
    cfg.dim, cfg.degree = 3, 1
    for a, e in enumerate((2048, 1024, 1024)):
        cfg.elems[a] = e
    free_before = torch.cuda.mem_get_info()[0]
    with pytest.raises(nat.NdgError) as ei:
        nat.ndg_create_ex(cfg)
    assert ei.value.status == nat.NDG_EINVAL and "2^31" in str(ei.value)
    assert torch.cuda.mem_get_info()[0] >= free_before - (64 << 20)


def test_a_zero_step_call_changes_nothing():
    p = orc.Problem(dim=2, degree=4, elems=(3, 2, 1), equation=1, flux=1)
    U = initial(p)
    s = Solver(2, 4, (3, 2), equation=1, flux=1)
    s.set_state(U)
    s.step(1e-3, 0, 4)
    nat.ndg_step_split(s.ctx, 1e-3, 0, 4)
    assert np.array_equal(s.get_state(), U)
    n = nat.ndg_norms(s.ctx)
    assert n.steps == 0 and n.t == 0.0
    s.close()
