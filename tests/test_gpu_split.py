"""The RK stage in split form (one volume-term and one surface-term kernel per axis, then the
stage-update kernel, over a right-hand-side array in global memory) against the fused stage
kernel: the same operations in the same order, so the states agree bit for bit -- FP64 and FP32,
advection and isothermal Euler, 1D/2D/3D, RK3/RK4/RK6, both thread mappings, the bulk-copy and
the paired-FP32 3D classes, an advection velocity with a zero component (no flux along that axis)
and one with a negative component (the upwind face on the other side)."""
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

CASES = [(1, 1, (9,), 0), (1, 4, (7,), 1), (1, 7, (5,), 0),
         (2, 2, (5, 3), 1), (2, 3, (6, 5), 0), (2, 5, (4, 3), 1), (2, 6, (5, 3), 0), (2, 7, (4, 3), 1),
         (3, 2, (3, 2, 3), 0), (3, 3, (2, 3, 2), 1), (3, 4, (3, 2, 2), 1), (3, 5, (3, 2, 3), 1),
         (3, 5, (2, 3, 2), 0), (3, 6, (2, 2, 3), 1), (3, 7, (2, 2, 3), 1), (3, 7, (2, 3, 2), 0)]
VELOCITIES = [(0.7, -0.4, 0.3), (-0.5, 0.0, 0.8)]


@pytest.mark.parametrize("dim,N,E,eq", CASES)
def test_split_stage_equals_the_fused_stage_bitwise(dim, N, E, eq):
    flux = 0 if eq == 0 else 1
    velocities = VELOCITIES if eq == 0 else VELOCITIES[:1]
    for vel in velocities:
        kw = dict(equation=eq, flux=flux, length=(1.0, 0.8, 1.2), velocity=vel)
        p = orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - dim), **kw)
        U = initial(p)
        dt = orc.stable_dt(p, U, 0.2)
        for dtype in ("f64", "f32"):
            for rk in (3, 4, 6):
                for kernel in (nat.NDG_KERNEL_LINE, nat.NDG_KERNEL_LINE_VAR):
                    epb = 0 if dim == 3 and N == 6 else 2  # 0: the library's pick (2 does not fit)
                    fused = Solver(dim, N, E, dtype=dtype, elems_per_block=epb, kernel=kernel, **kw)
                    split = Solver(dim, N, E, dtype=dtype, elems_per_block=epb, kernel=kernel, **kw)
                    fused.set_state(U)
                    split.set_state(U)
                    fused.step(dt, 2, rk)
                    nat.ndg_step_split(split.ctx, dt, 2, rk)
                    a, b = fused.get_state(), split.get_state()
                    assert np.array_equal(a, b), (vel, dtype, rk, kernel, np.max(np.abs(a - b)))
                    fused.close()
                    split.close()
                ref = orc.step(p, U.astype(np.float32).astype(np.float64) if dtype == "f32" else U, dt, 2, rk)
                assert rel_l2(b, ref) < (F64_TOL if dtype == "f64" else 2 * F32_TOL), (vel, dtype, rk)


def test_split_stage_rejects_the_float_float_and_exact_mass_classes():
    for kw in (dict(dtype="f64ff"), dict(dtype="f64", mass=nat.NDG_MASS_EXACT)):
        s = Solver(2, 3, (4, 3), equation=1, flux=1, **kw)
        p = orc.Problem(dim=2, degree=3, elems=(4, 3, 1), equation=1, flux=1)
        s.set_state(initial(p))
        with pytest.raises(nat.NdgError) as ei:
            nat.ndg_step_split(s.ctx, 1e-3, 1, 4)
        assert ei.value.status == nat.NDG_EINVAL
        s.close()


def test_split_stage_time_and_step_count_advance_like_ndg_step():
    p = orc.Problem(dim=2, degree=4, elems=(4, 4, 1), equation=0, flux=0, velocity=(1.0, 0.5, 0.0))
    s = Solver(2, 4, (4, 4), velocity=(1.0, 0.5, 0.0))
    s.set_state(initial(p))
    nat.ndg_step_split(s.ctx, 1e-3, 3, 4)
    nat.ndg_step_split(s.ctx, 1e-3, 0, 4)
    n = nat.ndg_norms(s.ctx)
    assert n.steps == 3 and abs(n.t - 3e-3) < 1e-15
    s.close()
