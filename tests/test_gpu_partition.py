"""Domain decomposition with a face-trace halo exchange (ndg_partition_*), emulated on one GPU:
the partitioned solve must equal the unpartitioned one bit for bit (same per-element arithmetic;
only where the neighbour's trace is read from changes), for uneven splits in 1D/2D/3D, in FP64,
FP32 and with the float-float contraction (its own kernels for 3D Euler at degrees 5 and 7)."""
import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05254_b300 import native as nat  # noqa: E402
from paper_2510_05254_b300.solver import Solver  # noqa: E402
from tests.test_gpu_parity import initial  # noqa: E402

CASES = [(1, 4, (11,), 1, (4,)), (2, 5, (12, 9), 0, (3, 2)), (2, 7, (10, 7), 1, (2, 3)),
         (3, 3, (4, 6, 5), 1, (2, 3, 2)), (3, 2, (5, 4, 3), 0, (1, 2, 3)), (2, 3, (9, 8), 1, (2, 3)),
         (3, 5, (4, 3, 5), 1, (2, 1, 2)), (3, 7, (3, 4, 3), 1, (2, 2, 1)),
         (3, 7, (2, 3, 4), 0, (1, 1, 2))]


def _cfg(dim, N, E, eq, dtype):
    cfg = nat.ndg_config_init()
    cfg.dim, cfg.degree = dim, N
    for a in range(3):
        cfg.elems[a] = E[a] if a < dim else 1
        cfg.length[a] = (1.0, 0.8, 1.2)[a]
    cfg.velocity[0], cfg.velocity[1], cfg.velocity[2] = 0.7, -0.4, 0.3
    cfg.equation, cfg.flux = eq, (0 if eq == 0 else 1)
    cfg.dtype = {"f64": nat.NDG_F64, "f32": nat.NDG_F32, "f64ff": nat.NDG_F64_FF}[dtype]
    return cfg


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64ff"])
@pytest.mark.parametrize("rk", [4, 6])
@pytest.mark.parametrize("dim,N,E,eq,parts", CASES)
def test_partitioned_equals_unpartitioned(dim, N, E, eq, parts, rk, dtype):
    p = orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - dim), equation=eq, flux=0 if eq == 0 else 1,
                    length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3))
    U = initial(p).astype(np.float32 if dtype == "f32" else np.float64)
    dt = orc.stable_dt(p, U.astype(np.float64), 0.2)
    s = Solver(dim, N, E, equation=eq, length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3), dtype=dtype)
    s.set_state(U)
    s.step(dt, 3, rk)
    ref = s.get_state()
    whole = s.norms()
    part = nat.ndg_partition_create(_cfg(dim, N, E, eq, dtype), parts)
    try:
        covered = 0
        for i in range(int(np.prod(parts))):
            off, cnt = nat.ndg_partition_info(part, i)
            assert all(0 <= off[a] and off[a] + cnt[a] <= (E[a] if a < dim else 1) for a in range(3))
            covered += int(np.prod(cnt))
        assert covered == int(np.prod(E))
        nat.ndg_partition_set_state(part, U.ctypes.data, U.nbytes, False)
        nat.ndg_partition_step(part, dt, 1, rk)
        nat.ndg_partition_step(part, dt, 2, rk)
        out = np.empty_like(U)
        nat.ndg_partition_get_state(part, out.ctypes.data, out.nbytes, False)
        assert np.array_equal(out, ref)
        pn = nat.ndg_partition_norms(part)
        assert abs(pn.l2 - whole["l2"]) < 1e-12 * whole["l2"]
        np.testing.assert_allclose(list(pn.integral)[:p.nvar], whole["integral"], rtol=1e-12, atol=1e-13)
        assert pn.steps == 3
    finally:
        nat.ndg_partition_destroy(part)


def test_partition_argument_errors():
    cfg = _cfg(2, 3, (4, 4), 0, "f64")
    with pytest.raises(nat.NdgError) as ei:
        nat.ndg_partition_create(cfg, (5, 1))
    assert ei.value.status == nat.NDG_EINVAL
    part = nat.ndg_partition_create(cfg, (2, 2))
    try:
        with pytest.raises(nat.NdgError) as ei:
            nat.ndg_partition_step(part, 0.01, 1, 4)
        assert ei.value.status == nat.NDG_ESTATE
    finally:
        nat.ndg_partition_destroy(part)


@pytest.mark.parametrize("dim,N,E,eq,parts", [(2, 7, (6, 5), 1, (2, 2)), (3, 5, (4, 3, 4), 1, (2, 1, 2))])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_partitioned_exact_mass(dim, N, E, eq, parts, dtype):
    """The exact-mass variant through the partition emulation: bitwise the unpartitioned solve."""
    p = orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - dim), equation=eq, flux=1,
                    length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3), mass=orc.MASS_EXACT)
    U = initial(p).astype(np.float64 if dtype == "f64" else np.float32)
    dt = 0.5 * orc.stable_dt(p, U.astype(np.float64), 0.2)
    s = Solver(dim, N, E, equation=eq, length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3), dtype=dtype,
               mass=nat.NDG_MASS_EXACT)
    s.set_state(U)
    s.step(dt, 2, 4)
    ref = s.get_state()
    cfg = _cfg(dim, N, E, eq, dtype)
    cfg.mass = nat.NDG_MASS_EXACT
    part = nat.ndg_partition_create(cfg, parts)
    try:
        nat.ndg_partition_set_state(part, U.ctypes.data, U.nbytes, False)
        nat.ndg_partition_step(part, dt, 2, 4)
        out = np.empty_like(U)
        nat.ndg_partition_get_state(part, out.ctypes.data, out.nbytes, False)
        assert np.array_equal(out, ref)
    finally:
        nat.ndg_partition_destroy(part)
