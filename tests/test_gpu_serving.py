"""Serving pool (ndg_pool_*): continuous batching of independent solves under a memory budget.
Each solve's result inside the mix must equal, bit for bit, its result computed alone through
ndg_step (same kernels, same per-element arithmetic)."""
import time

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2510_05254_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05254_b300 import native as nat  # noqa: E402
from paper_2510_05254_b300.solver import Solver  # noqa: E402


def _spec_state(dim, N, E, eq, dtype, seed):
    p = orc.Problem(dim=dim, degree=N, elems=tuple(E) + (1,) * (3 - len(E)), equation=eq,
                    flux=0 if eq == 0 else 1, velocity=(1.0, 0.5, 0.25))
    X = orc.node_coords(p)
    if eq == 0:
        U = inputs.gaussian_noise(X, seed=seed) if dim == 2 else inputs.sine(X)
    else:
        U = inputs.euler_shear(X, seed=seed) if dim == 2 else inputs.taylor_green(X)
    dt = orc.stable_dt(p, U, 0.1)
    return U.astype(np.float64 if dtype == "f64" else np.float32), dt


def _cfg(dim, N, E, eq, dtype):
    cfg = nat.ndg_config_init()
    cfg.dim, cfg.degree = dim, N
    for a in range(3):
        cfg.elems[a] = E[a] if a < dim else 1
    cfg.velocity[0], cfg.velocity[1], cfg.velocity[2] = 1.0, 0.5, 0.25
    cfg.equation, cfg.flux = eq, (0 if eq == 0 else 1)
    cfg.dtype = nat.NDG_F64 if dtype == "f64" else nat.NDG_F32
    return cfg


def _alone(dim, N, E, eq, dtype, U, dt, nsteps, rk=4):
    s = Solver(dim, N, E, equation=eq, dtype=dtype, velocity=(1.0, 0.5, 0.25))
    s.set_state(U)
    s.step(dt, nsteps, rk)
    out = s.get_state()
    s.close()
    return out


SPECS = [(2, 3, (16, 16), 0, "f64", 30), (2, 7, (24, 20), 1, "f64", 25), (2, 5, (40, 40), 0, "f32", 40),
         (2, 7, (16, 16), 0, "f64", 12), (2, 3, (33, 17), 1, "f32", 35), (3, 2, (4, 5, 3), 1, "f64", 20),
         (2, 5, (20, 20), 1, "f64", 50), (1, 7, (50,), 0, "f32", 10)]


def test_pool_results_bitwise_equal_to_solo():
    pool = nat.ndg_pool_create(8 << 30)
    tickets = []
    try:
        for i, (dim, N, E, eq, dtype, nsteps) in enumerate(SPECS):
            U, dt = _spec_state(dim, N, E, eq, dtype, seed=100 + i)
            t = nat.ndg_pool_submit(pool, _cfg(dim, N, E, eq, dtype), U.ctypes.data, U.nbytes, 4, dt, nsteps)
            tickets.append((t, U, dt))
        for (t, U, dt), (dim, N, E, eq, dtype, nsteps) in zip(tickets, SPECS):
            out = np.empty_like(U)
            rc, st = nat.ndg_pool_poll(pool, t, out.ctypes.data, out.nbytes, 60.0)
            assert rc == nat.NDG_OK
            assert st.steps == nsteps and st.latency_s > 0 and st.done_s >= st.admit_s >= st.submit_s
            assert np.array_equal(out, _alone(dim, N, E, eq, dtype, U, dt, nsteps))
        s = nat.ndg_pool_status(pool)
        assert s["finished"] == len(SPECS) and s["bytes_in_use"] == 0
    finally:
        nat.ndg_pool_destroy(pool)


def test_pool_budget_is_never_exceeded_and_late_arrivals_are_admitted():
    U, dt = _spec_state(2, 5, (32, 32), 1, "f64", seed=7)
    need = U.nbytes * 4  # RK4 holds four state-sized arrays
    pool = nat.ndg_pool_create(int(2.5 * need))  # room for two at a time
    try:
        tks = [nat.ndg_pool_submit(pool, _cfg(2, 5, (32, 32), 1, "f64"), U.ctypes.data, U.nbytes, 4, dt, 60)
               for _ in range(5)]
        time.sleep(0.05)
        late = nat.ndg_pool_submit(pool, _cfg(2, 5, (32, 32), 1, "f64"), U.ctypes.data, U.nbytes, 4, dt, 15)
        ref = _alone(2, 5, (32, 32), 1, "f64", U, dt, 60)
        for t in tks:
            out = np.empty_like(U)
            rc, _ = nat.ndg_pool_poll(pool, t, out.ctypes.data, out.nbytes, 60.0)
            assert rc == nat.NDG_OK and np.array_equal(out, ref)
        out = np.empty_like(U)
        rc, st = nat.ndg_pool_poll(pool, late, out.ctypes.data, out.nbytes, 60.0)
        assert rc == nat.NDG_OK and st.steps == 15
        assert np.array_equal(out, _alone(2, 5, (32, 32), 1, "f64", U, dt, 15))
        s = nat.ndg_pool_status(pool)
        assert s["peak_bytes"] <= int(2.5 * need) and s["peak_bytes"] >= need
    finally:
        nat.ndg_pool_destroy(pool)


def test_pool_status_codes():
    U, dt = _spec_state(2, 7, (64, 64), 0, "f64", seed=3)
    pool = nat.ndg_pool_create(10 << 20)  # 10 MiB: the 64^2 solve (8.4 MB) fits, 128^2 does not
    try:
        with pytest.raises(nat.NdgError) as ei:  # alone larger than the budget
            big, _ = _spec_state(2, 7, (128, 128), 0, "f64", seed=3)
            nat.ndg_pool_submit(pool, _cfg(2, 7, (128, 128), 0, "f64"), big.ctypes.data, big.nbytes, 4, dt, 1)
        assert ei.value.status == nat.NDG_ENOMEM
        with pytest.raises(nat.NdgError) as ei:
            nat.ndg_pool_submit(pool, _cfg(2, 7, (64, 64), 0, "f64"), U.ctypes.data, U.nbytes - 8, 4, dt, 1)
        assert ei.value.status == nat.NDG_EINVAL
        t = nat.ndg_pool_submit(pool, _cfg(2, 7, (64, 64), 0, "f64"), U.ctypes.data, U.nbytes, 4, dt, 20000)
        rc, _ = nat.ndg_pool_poll(pool, t, None, 0, 0.0)
        assert rc == nat.NDG_EAGAIN
        rc, _ = nat.ndg_pool_poll(pool, t, None, 0, 0.001)
        assert rc == nat.NDG_ETIMEOUT
        rc, st = nat.ndg_pool_poll(pool, t, None, 0, 120.0)
        assert rc == nat.NDG_OK and st.steps == 20000
        with pytest.raises(nat.NdgError) as ei:
            nat.ndg_pool_poll(pool, t, None, 0, 0.0)  # forgotten after the successful poll
        assert ei.value.status == nat.NDG_EINVAL
    finally:
        nat.ndg_pool_destroy(pool)


def test_pool_keeps_exact_and_lumped_mass_apart():
    """Solves that differ only in the mass matrix are separate kernel classes in the pool: each
    result equals its own solve alone."""
    pool = nat.ndg_pool_create(4 << 30)
    try:
        U, dt = _spec_state(2, 5, (20, 16), 1, "f64", seed=7)
        g = np.random.default_rng(3)
        U = U + 0.01 * g.standard_normal(U.shape)  # faces jump: the two lifts differ
        tickets = []
        for mass in (nat.NDG_MASS_EXACT, nat.NDG_MASS_LUMPED, nat.NDG_MASS_EXACT):
            cfg = _cfg(2, 5, (20, 16), 1, "f64")
            cfg.mass = mass
            tickets.append((nat.ndg_pool_submit(pool, cfg, U.ctypes.data, U.nbytes, 4, dt, 15), mass))
        for t, mass in tickets:
            out = np.empty_like(U)
            rc, _ = nat.ndg_pool_poll(pool, t, out.ctypes.data, out.nbytes, 60.0)
            assert rc == nat.NDG_OK
            s = Solver(2, 5, (20, 16), equation=1, velocity=(1.0, 0.5, 0.25), mass=mass)
            s.set_state(U)
            s.step(dt, 15, 4)
            assert np.array_equal(out, s.get_state())
            s.close()
    finally:
        nat.ndg_pool_destroy(pool)
