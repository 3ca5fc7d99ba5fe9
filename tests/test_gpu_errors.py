"""The bounded wait of the bulk-copy stage kernels, made to run out without any fault.

The FP32 stage kernels of degree 5 (2D and 3D) and of degree 7 (3D) copy their element tiles
into shared memory by bulk copies completed on an mbarrier, and every thread's wait on that
barrier gives up after a bounded number of polls.  The test switch ndg_debug_stall_copies arms
the barrier with the tile's byte count but issues no copy, so the phase never completes and the
wait runs out; nothing is left in flight when the kernel returns.  The host must then report
NDG_ECUDA from every synchronising call of each solve the failed launch served -- also after the
work list has been uploaded again (a new dt), which must not wipe the flag -- until a new state
is set, after which stepping works and matches the oracle again."""
import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05254_b300 import native as nat  # noqa: E402
from paper_2510_05254_b300.solver import Batch, Solver  # noqa: E402
from tests.test_gpu_parity import F32_TOL, F64_TOL, initial, rel_l2  # noqa: E402

POLLS = 1 << 12  # polls before a stalled wait gives up (the default limit is 2^22)

# FP32 isothermal Euler classes whose tiles arrive by bulk copies: 3D degree 5 (one copy per
# element and variable), 3D degree 7 (one per z-plane), 2D degree 5 (one per variable)
BULK_CASES = [(3, 5, (3, 2, 3)), (3, 7, (2, 2, 2)), (2, 5, (4, 3))]


def _problem(dim, N, E, eq=1):
    return orc.Problem(dim=dim, degree=N, elems=tuple(E) + (1,) * (3 - dim), equation=eq, flux=1 if eq else 0)


def _raises_ecuda(fn, *args):
    with pytest.raises(nat.NdgError) as ei:
        fn(*args)
    assert ei.value.status == nat.NDG_ECUDA, ei.value
    assert "wait limit" in str(ei.value), ei.value


@pytest.fixture(autouse=True)
def _switch_off_afterwards():
    yield
    nat.ndg_debug_stall_copies(0)


@pytest.mark.parametrize("dim,N,E", BULK_CASES)
def test_context_reports_the_wait_that_ran_out_until_a_new_state(dim, N, E):
    p = _problem(dim, N, E)
    U = initial(p).astype(np.float32)
    dt = orc.stable_dt(p, U.astype(np.float64), 0.2)
    s = Solver(dim, N, E, equation=1, dtype="f32", elems_per_block=2)
    s.set_state(U)
    nat.ndg_debug_stall_copies(POLLS)
    s.step(dt, 1, 4)  # the first step with this dt uploads the work list: with the stall
    nat.ndg_debug_stall_copies(0)
    _raises_ecuda(s.synchronize)
    # a new dt uploads the work list again (now without the stall): the flag survives it
    s.step(0.5 * dt, 1, 4)
    _raises_ecuda(s.synchronize)
    _raises_ecuda(s.get_state)
    _raises_ecuda(nat.ndg_norms, s.ctx)
    # a new state clears the flag; the kernels run normally again
    s.set_state(U)
    s.step(dt, 1, 4)
    s.synchronize()
    ref = orc.step(p, U.astype(np.float64), dt, 1, 4)
    assert rel_l2(s.get_state(), ref) < F32_TOL
    s.close()


def test_batch_flags_the_members_of_the_failed_launch_only():
    pa, pb = _problem(3, 5, (3, 2, 3)), _problem(2, 3, (4, 3))
    Ua, Ub = initial(pa).astype(np.float32), initial(pb)
    dta = orc.stable_dt(pa, Ua.astype(np.float64), 0.2)
    dtb = orc.stable_dt(pb, Ub, 0.2)
    a = Solver(3, 5, (3, 2, 3), equation=1, dtype="f32", elems_per_block=2)  # bulk-copy class
    b = Solver(2, 3, (4, 3), equation=1, dtype="f64")                       # no bulk copies
    a.set_state(Ua)
    b.set_state(Ub)
    batch = Batch([a, b])
    nat.ndg_debug_stall_copies(POLLS)
    batch.step([dta, dtb], 1, 4)  # the batch uploads its work lists on every step
    nat.ndg_debug_stall_copies(0)
    _raises_ecuda(a.synchronize)
    b.synchronize()
    assert rel_l2(b.get_state(), orc.step(pb, Ub, dtb, 1, 4)) < F64_TOL
    # the next batch step runs normally; the failed member stays flagged until its new state
    batch.step([dta, dtb], 1, 4)
    _raises_ecuda(a.get_state)
    a.set_state(Ua)
    b.set_state(Ub)
    batch.step([dta, dtb], 1, 4)
    a.synchronize()
    assert rel_l2(a.get_state(), orc.step(pa, Ua.astype(np.float64), dta, 1, 4)) < F32_TOL
    batch.close()
    a.close()
    b.close()


def test_pool_reports_the_solve_whose_launch_failed():
    p = _problem(3, 5, (3, 2, 3))
    U = initial(p).astype(np.float32)
    dt = orc.stable_dt(p, U.astype(np.float64), 0.2)
    cfg = nat.ndg_config_init()
    cfg.dim, cfg.degree, cfg.equation, cfg.flux, cfg.dtype = 3, 5, 1, 1, nat.NDG_F32
    for a, e in enumerate((3, 2, 3)):
        cfg.elems[a] = e
    out = np.empty_like(U)
    pool = nat.ndg_pool_create(1 << 30)
    try:
        nat.ndg_debug_stall_copies(POLLS)
        t = nat.ndg_pool_submit(pool, cfg, U.ctypes.data, U.nbytes, 4, dt, 3)
        with pytest.raises(nat.NdgError) as ei:
            nat.ndg_pool_poll(pool, t, out.ctypes.data, out.nbytes, 120.0)
        assert ei.value.status == nat.NDG_ECUDA and "wait limit" in str(ei.value)
        nat.ndg_debug_stall_copies(0)
        # a later solve of the same class is admitted with the switch off and succeeds
        t = nat.ndg_pool_submit(pool, cfg, U.ctypes.data, U.nbytes, 4, dt, 3)
        rc, _ = nat.ndg_pool_poll(pool, t, out.ctypes.data, out.nbytes, 120.0)
        assert rc == nat.NDG_OK
        assert rel_l2(out, orc.step(p, U.astype(np.float64), dt, 3, 4)) < 4 * F32_TOL
    finally:
        nat.ndg_pool_destroy(pool)


def test_stall_switch_rejects_negative_polls():
    with pytest.raises(nat.NdgError) as ei:
        nat.ndg_debug_stall_copies(-1)
    assert ei.value.status == nat.NDG_EINVAL
