"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances: FP64 within 1e-12 relative L2 per step (after 1 step and after a few steps); FP32
within the per-case bound stated here (FP32 state rounding, ~1e-7 relative per stage, amplified
by the operator norm dt*|L| ~ CFL)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2510_05254_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05254_b300 import native as nat  # noqa: E402
from paper_2510_05254_b300.solver import Solver, Batch  # noqa: E402

F64_TOL = 1e-12
F32_TOL = 2e-6


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a, np.float64) - b).ravel()) / np.linalg.norm(b.ravel()))


def make(dim, N, E, eq, dtype="f64", epb=0, length=(1.0, 1.0, 1.0), velocity=(1.0, 0.5, 0.25), c=1.0):
    E = tuple(E)
    flux = 0 if eq == 0 else 1
    p = orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - len(E)), equation=eq, flux=flux,
                    length=length, velocity=velocity, sound_speed=c)
    s = Solver(dim, N, E, equation=eq, flux=flux, dtype=dtype, length=length, velocity=velocity,
               sound_speed=c, elems_per_block=epb)
    return p, s


def initial(p, seed=3):
    """Smooth random-mode state plus a small seeded perturbation (so element faces jump)."""
    X = orc.node_coords(p)
    if p.equation == 0:
        U = np.zeros(p.shape)
        for a in range(p.dim):
            U[0] += inputs.random_modes(X[a:a + 1] / p.length[a], nk=3, seed=seed + a)[0]
    else:
        U = np.zeros(p.shape)
        U[0] = 1.0 + 0.1 * np.sin(2 * math.pi * X[0] / p.length[0])
        for a in range(p.dim):
            U[1 + a] = 0.2 * np.cos(2 * math.pi * (X[a] / p.length[a] + 0.1 * (a + 1)))
    U += 1e-3 * inputs.random_state(p.shape, seed + 100)
    return U


def check(p, s, U, dt, nsteps, rk, tol):
    s.set_state(U)
    ref = U.copy()
    worst = 0.0
    for k in range(nsteps):
        s.step(dt, 1, rk)
        got = s.get_state()
        ref = orc.step(p, ref, dt, 1, rk)
        err = rel_l2(got, ref)
        worst = max(worst, err)
        assert err < tol, (k, err)
        # next step from the same state on both sides: the tolerance is per step
        s.set_state(ref)
    return worst


CASES_2D = [(N, eq) for N in range(1, 8) for eq in (0, 1)]


@pytest.mark.parametrize("N,eq", CASES_2D)
def test_2d_all_degrees_ragged_tiles(N, eq):
    # 5 x 3 = 15 elements in tiles of 4: three full tiles and a ragged one, neighbours both
    # inside and outside the tile along x, always outside along y
    p, s = make(2, N, (5, 3), eq, epb=4, length=(1.0, 0.7, 1.0), velocity=(0.9, -0.6, 0))
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    check(p, s, U, dt, 2, 4, F64_TOL)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("eq", [0, 1])
def test_1d(N, eq):
    p, s = make(1, N, (9,), eq, epb=4, velocity=(-0.8, 0, 0))
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    check(p, s, U, dt, 2, 4, F64_TOL)


@pytest.mark.parametrize("N,eq", [(1, 0), (2, 0), (3, 0), (5, 0), (7, 0), (1, 1), (2, 1), (3, 1), (5, 1)])
def test_3d(N, eq):
    p, s = make(3, N, (3, 2, 3), eq, epb=5, length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3))
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    check(p, s, U, dt, 2, 4, F64_TOL)


@pytest.mark.parametrize("rk", [3, 4, 6])
@pytest.mark.parametrize("dim,N,E,eq", [(2, 5, (4, 3), 0), (2, 4, (3, 3), 1), (3, 3, (2, 2, 3), 1)])
def test_runge_kutta_schemes(rk, dim, N, E, eq):
    p, s = make(dim, N, E, eq, epb=3)
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    check(p, s, U, dt, 3, rk, F64_TOL)


def test_oversized_tile_is_rejected():
    # 2D Euler at degree 7 in FP64 needs 8 x 72 x 8 B of shared memory per element: 64 do not fit
    with pytest.raises(nat.NdgError) as ei:
        make(2, 7, (9, 8), 1, epb=64)
    assert ei.value.status == nat.NDG_EINVAL
    # 8 elements x 36 lines x 4 variables = 1152 threads exceed 1024
    with pytest.raises(nat.NdgError) as ei:
        Solver(3, 5, (2, 2, 3), equation=1, elems_per_block=8, kernel=nat.NDG_KERNEL_LINE_VAR, dtype="f32")
    assert ei.value.status == nat.NDG_EINVAL


@pytest.mark.parametrize("epb", [1, 2, 3, 7, 16, 24])
def test_tile_size_does_not_change_results_bitwise(epb):
    p, s = make(2, 7, (9, 7), 1, epb=epb)
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    s.set_state(U)
    s.step(dt, 3, 4)
    got = s.get_state()
    p2, s2 = make(2, 7, (9, 7), 1, epb=5)
    s2.set_state(U)
    s2.step(dt, 3, 4)
    assert np.array_equal(got, s2.get_state())


# (2, 7) and (2, 3) take the FP32 kernel's 16-byte-aligned 2D layout, (2, 5) and (3, 5) its
# unpadded layout with bulk tile copies, (3, 7) its plane-padded 3D layout with one bulk copy per
# plane; the others the padded layout
@pytest.mark.parametrize("dim,N,E,eq", [(1, 3, (11,), 0), (2, 7, (6, 5), 0), (2, 7, (6, 5), 1), (2, 5, (5, 4), 1),
                                        (2, 3, (7, 5), 1), (3, 3, (3, 3, 2), 1), (3, 5, (3, 2, 3), 1),
                                        (3, 5, (2, 3, 3), 0), (3, 7, (3, 2, 3), 1), (3, 7, (2, 3, 2), 0)])
def test_fp32_path(dim, N, E, eq):
    p, s = make(dim, N, E, eq, dtype="f32", epb=4)
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    s.set_state(U)
    s.step(dt, 1, 4)
    ref = orc.step(p, U.astype(np.float32).astype(np.float64), dt, 1, 4)
    assert rel_l2(s.get_state(), ref) < F32_TOL
    s.step(dt, 9, 4)
    ref = orc.step(p, ref, dt, 9, 4)
    assert rel_l2(s.get_state(), ref) < 10 * F32_TOL
    # the other schemes' stage plans (RK3: ACC accumulation; RK6: stored slopes), ragged tiles
    for rk in (3, 6):
        p3, s3 = make(dim, N, E, eq, dtype="f32", epb=3)
        s3.set_state(U)
        s3.step(dt, 2, rk)
        ref = orc.step(p3, U.astype(np.float32).astype(np.float64), dt, 2, rk)
        assert rel_l2(s3.get_state(), ref) < 2 * F32_TOL


def test_config1_one_revolution_matches_oracle():
    """1D advection, E = 64, N = 3, sin(2 pi x), upwind, RK4, CFL 0.1, integrated to t = 1."""
    p, s = make(1, 3, (64,), 0, velocity=(1.0, 0, 0))
    X = orc.node_coords(p)
    U0 = inputs.sine(X)
    dt = orc.stable_dt(p, U0, 0.1)
    nsteps = int(math.ceil(1.0 / dt))
    dt = 1.0 / nsteps
    s.set_state(U0)
    s.step(dt, nsteps, 4)
    got = s.get_state()
    ref = orc.step(p, U0, dt, nsteps, 4)
    assert rel_l2(got, ref) < 1e-11
    n = s.norms(U0)
    assert abs(s.norms()["t"] - 1.0) < 1e-12
    assert n["l2"] < 1e-7 and abs(n["l2"] - orc.norms(p, ref, U0)["l2"]) < 1e-12


def per_element_check(got, ref, tol):
    """Every element on its own: the largest |got - ref| over an element's nodes against tol times
    the largest |ref| of the whole state (an error confined to one element cannot hide in a norm
    over millions of values)."""
    err = np.abs(np.asarray(got, np.float64) - ref).max(axis=-1)  # (variables, elements)
    bound = tol * np.abs(ref).max()
    v, e = np.unravel_index(int(np.argmax(err)), err.shape)
    assert err[v, e] < bound, ("variable", int(v), "element", int(e), float(err[v, e]), bound)


def test_config2_full_size_one_step_fp64_and_fp32():
    """2D advection, 256^2 elements of degree 7 (4.2M DOF), Gaussian + Fourier noise, RK4:
    one full step compared with the oracle, as a whole and element by element."""
    p = orc.Problem(dim=2, degree=7, elems=(256, 256, 1), equation=0, flux=0, velocity=(1.0, 0.5, 0))
    X = orc.node_coords(p)
    U0 = inputs.gaussian_noise(X)
    dt = orc.stable_dt(p, U0, 0.1)
    ref = orc.step(p, U0, dt, 1, 4)
    for dtype, tol in (("f64", F64_TOL), ("f32", F32_TOL)):
        s = Solver(2, 7, (256, 256), velocity=(1.0, 0.5, 0), dtype=dtype)
        s.set_state(U0)
        s.step(dt, 1, 4)
        got = s.get_state()
        assert rel_l2(got, ref) < tol, dtype
        per_element_check(got, ref, tol)
        s.close()


def _patch_check(dim, N, E, eq, U0, dt, rk, samples, velocity=(1.0, 0.5, 0.25), tol=F64_TOL,
                 dtype="f64"):
    """Full-size GPU step; the oracle recomputes sampled elements on a periodic patch of
    (2S+1)^dim elements around each (S = number of stages: the dependency cone of one step)."""
    s = Solver(dim, N, E, equation=eq, flux=0 if eq == 0 else 1, velocity=velocity, dtype=dtype)
    s.set_state(U0)
    s.step(dt, 1, rk)
    got = s.get_state()
    s.close()
    S = {3: 3, 4: 4, 6: 7}[rk]
    W = 2 * S + 1
    n = N + 1
    nv = U0.shape[0]
    Eg = list(E)
    Uf = U0.reshape([nv] + Eg[::-1] + [n ** dim])
    Gf = got.reshape([nv] + Eg[::-1] + [n ** dim])
    p = orc.Problem(dim=dim, degree=N, elems=(W,) * dim + (1,) * (3 - dim), equation=eq,
                    flux=0 if eq == 0 else 1, length=tuple(W / E[a] for a in range(dim)) + (1.0,) * (3 - dim),
                    velocity=velocity)
    worst = 0.0
    for (idx) in samples:
        rng = [np.arange(idx[a] - S, idx[a] + S + 1) % E[a] for a in range(dim)]
        patch = Uf[np.ix_(range(nv), *[r for r in rng[::-1]], range(n ** dim))]
        out = orc.step(p, patch.reshape(nv, -1, n ** dim), dt, 1, rk).reshape(patch.shape)
        center = tuple([slice(None)] + [S] * dim + [slice(None)])
        ref = out[center]
        g = Gf[tuple([slice(None)] + [idx[a] for a in range(dim)][::-1] + [slice(None)])]
        err = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
        worst = max(worst, err)
        assert err < tol, (idx, err)
    return worst


def test_config3_full_size_sampled():
    """2D isothermal Euler, 512^2 elements of degree 7 (50M DOF), one RK4 step on the GPU;
    sampled elements (corners, edges, interior) recomputed by the oracle on patches."""
    p = orc.Problem(dim=2, degree=7, elems=(512, 512, 1), equation=1, flux=1)
    X = orc.node_coords(p)
    U0 = inputs.euler_shear(X)
    del X
    dt = orc.stable_dt(p, U0, 0.1)
    samples = [(0, 0), (511, 511), (0, 300), (257, 0), (123, 456), (511, 7)]
    _patch_check(2, 7, (512, 512), 1, U0, dt, 4, samples)


def test_config4_full_size_sampled_rk4_rk6():
    """3D isothermal Euler, 64^3 elements of degree 5 (226M DOF), Taylor-Green velocity; one
    step of RK4 and of RK6, sampled elements recomputed by the oracle on patches."""
    p = orc.Problem(dim=3, degree=5, elems=(64, 64, 64), equation=1, flux=1)
    X = orc.node_coords(p)
    U0 = inputs.taylor_green(X)
    del X
    dt = orc.stable_dt(p, U0, 0.1)
    _patch_check(3, 5, (64, 64, 64), 1, U0, dt, 4, [(0, 0, 0), (63, 31, 5), (10, 63, 63)])
    _patch_check(3, 5, (64, 64, 64), 1, U0, dt, 6, [(0, 63, 0), (33, 2, 40)])
    # the float-float contraction at the FP64 bar (its own register-capped kernel at this degree)
    _patch_check(3, 5, (64, 64, 64), 1, U0, dt, 4, [(0, 0, 0), (40, 63, 17)], dtype="f64ff")


def test_norms_match_oracle():
    for dim, N, E, eq in [(2, 7, (6, 5), 0), (2, 4, (4, 4), 1), (3, 3, (2, 3, 2), 1), (1, 5, (7,), 0)]:
        p, s = make(dim, N, E, eq)
        U = initial(p)
        ref = U + 0.01 * inputs.random_state(p.shape, 9)
        s.set_state(U)
        a, b = s.norms(ref), orc.norms(p, U, ref)
        assert abs(a["l2"] - b["l2"]) < 1e-13 * max(1, b["l2"])
        assert abs(a["linf"] - b["linf"]) < 1e-15
        np.testing.assert_allclose(a["integral"], b["integral"], rtol=1e-13, atol=1e-14)
        a, b = s.norms(), orc.norms(p, U)
        assert abs(a["l2"] - b["l2"]) < 1e-13 * b["l2"]
        assert abs(s.stable_dt(0.3) - orc.stable_dt(p, U, 0.3)) < 1e-15


def test_mass_and_momentum_conserved_on_gpu():
    p, s = make(2, 7, (16, 16), 1)
    U = initial(p)
    s.set_state(U)
    m0 = s.norms()["integral"]
    s.step(orc.stable_dt(p, U, 0.1), 20, 4)
    m1 = s.norms()["integral"]
    np.testing.assert_allclose(m1, m0, rtol=0, atol=2e-14)


def test_grid_layout_round_trip():
    p, s = make(3, 2, (3, 4, 2), 1)
    U = initial(p)
    n = 3
    # natural grid [v][z][y][x] built by numpy from the element layout
    E = (3, 4, 2)
    G = U.reshape(4, E[2], E[1], E[0], n, n, n).transpose(0, 1, 4, 2, 5, 3, 6).reshape(4, E[2] * n, E[1] * n, E[0] * n)
    Gc = np.ascontiguousarray(G)
    nat.ndg_set_state(s.ctx, Gc.ctypes.data, Gc.nbytes, False, nat.NDG_LAYOUT_GRID)
    assert np.array_equal(s.get_state(), U)
    out = np.empty_like(Gc)
    nat.ndg_get_state(s.ctx, out.ctypes.data, out.nbytes, False, nat.NDG_LAYOUT_GRID)
    assert np.array_equal(out, Gc)


def test_device_state_round_trip_and_node_coords():
    p, s = make(2, 3, (4, 5), 0)
    U = torch.tensor(initial(p), device="cuda")
    s.set_state(U)
    assert torch.equal(s.get_state(device=True), U)
    np.testing.assert_allclose(s.node_coords(), orc.node_coords(p), rtol=0, atol=1e-15)


def test_batch_is_bitwise_identical_to_individual_solves():
    # two solves share a launch where their classes match (the float-float 3D degree-5 and 2D
    # degree-7 Euler classes included)
    specs = [(2, 7, (6, 5), 0, "f64"), (2, 3, (9, 4), 1, "f64"), (2, 7, (3, 3), 0, "f64"),
             (2, 5, (4, 4), 1, "f32"), (3, 2, (2, 3, 2), 1, "f64"), (3, 5, (2, 3, 2), 1, "f64ff"),
             (3, 5, (3, 2, 2), 1, "f64ff"), (2, 7, (3, 4), 1, "f64ff")]
    alone, batched, states, dts = [], [], [], []
    for dim, N, E, eq, dt_ in specs:
        p, s = make(dim, N, E, eq, dtype=dt_)
        U = initial(p)
        dt = orc.stable_dt(p, U, 0.2)
        s.set_state(U)
        s.step(dt, 4, 4)
        alone.append(s.get_state())
        s.close()
        _, sb = make(dim, N, E, eq, dtype=dt_)
        sb.set_state(U)
        batched.append(sb)
        dts.append(dt)
    b = Batch(batched)
    b.step(dts, 2, 4)
    b.step(dts, 2, 4)
    for a, sb in zip(alone, batched):
        assert np.array_equal(a, sb.get_state())
    b.close()


def test_autotune_restores_state_and_keeps_results():
    p, s = make(2, 7, (20, 20), 0)
    U = initial(p)
    s.set_state(U)
    best, ms = s.autotune(4)
    assert best >= 1 and ms > 0
    assert np.array_equal(s.get_state(), U)
    assert s.norms()["steps"] == 0
    dt = orc.stable_dt(p, U, 0.2)
    s.step(dt, 1, 4)
    assert rel_l2(s.get_state(), orc.step(p, U, dt, 1, 4)) < F64_TOL


def test_errors_on_gpu():
    p, s = make(2, 3, (4, 4), 0)
    with pytest.raises(nat.NdgError) as ei:
        s.step(0.01, 1, 4)
    assert ei.value.status == nat.NDG_ESTATE
    U = initial(p)
    s.set_state(U)
    with pytest.raises(nat.NdgError) as ei:
        s.step(-1.0, 1, 4)
    assert ei.value.status == nat.NDG_EINVAL
    with pytest.raises(nat.NdgError) as ei:
        s.step(0.01, 1, 5)
    assert ei.value.status == nat.NDG_EINVAL
    with pytest.raises(nat.NdgError) as ei:
        nat.ndg_set_state(s.ctx, U.ctypes.data, U.nbytes - 8, False)
    assert ei.value.status == nat.NDG_EINVAL
    bad = U.copy()
    bad[0, 3, 2] = np.nan
    s.set_state(bad)
    with pytest.raises(nat.NdgError) as ei:
        nat.ndg_norms(s.ctx)
    assert ei.value.status == nat.NDG_ENONFINITE
    assert s.norms()["nonfinite"] == 1


def test_torch_allocator_hook():
    """Device memory through torch's caching allocator (ndg_set_allocator)."""
    live = {}

    def alloc(nbytes, user, stream):
        ptr = torch.cuda.caching_allocator_alloc(nbytes, 0, stream)
        live[ptr] = nbytes
        return ptr

    def free(ptr, user, stream):
        live.pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    nat.ndg_set_allocator(alloc, free)
    try:
        p, s = make(2, 4, (5, 5), 1)
        assert len(live) >= 4
        U = initial(p)
        s.set_state(U)
        dt = orc.stable_dt(p, U, 0.2)
        s.step(dt, 1, 4)
        assert rel_l2(s.get_state(), orc.step(p, U, dt, 1, 4)) < F64_TOL
        s.close()
        assert not live
    finally:
        nat.ndg_set_allocator(None, None)


@pytest.mark.parametrize("kernel", [nat.NDG_KERNEL_LINE, nat.NDG_KERNEL_LINE_VAR])
@pytest.mark.parametrize("dim,N,E,eq", [(1, 4, (7,), 1), (2, 7, (5, 3), 0), (2, 6, (4, 3), 1), (2, 3, (6, 5), 1),
                                        (3, 2, (3, 2, 3), 1), (3, 5, (2, 2, 3), 0), (3, 3, (2, 3, 2), 1),
                                        (3, 5, (2, 3, 2), 1), (2, 7, (5, 4), 1), (3, 7, (2, 2, 3), 1)])
def test_both_kernel_mappings(kernel, dim, N, E, eq):
    """Thread per line (all variables) and thread per (line, variable): FP64 within 1e-12 per
    step (RK4 and RK6), FP32 within its tolerance, with tiles that leave a ragged end; and the
    two mappings agree bit for bit."""
    flux = 0 if eq == 0 else 1
    p = orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - len(E)), equation=eq, flux=flux,
                    length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3))
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    kw = dict(equation=eq, flux=flux, length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3))
    for rk in (4, 6):
        s = Solver(dim, N, E, elems_per_block=2, kernel=kernel, **kw)
        assert s.kernel == kernel
        check(p, s, U, dt, 2, rk, F64_TOL)
    # FP32 with every scheme: the stage plans with ACC accumulation (RK3) and stored slopes (RK6)
    for dtype, rks in (("f64", (4,)), ("f32", (3, 4, 6))):
        for rk in rks:
            outs = []
            for kern in (nat.NDG_KERNEL_LINE, nat.NDG_KERNEL_LINE_VAR):
                s = Solver(dim, N, E, elems_per_block=2, kernel=kern, dtype=dtype, **kw)
                s.set_state(U)
                s.step(dt, 2, rk)
                outs.append(s.get_state())
            assert np.array_equal(outs[0], outs[1]), (dtype, rk)
            if dtype == "f32" and rk == 4:
                ref = orc.step(p, U.astype(np.float32).astype(np.float64), dt, 2, 4)
                assert rel_l2(outs[1], ref) < 2 * F32_TOL


# ---- FP64 state with the float-float contraction (NDG_F64_FF): the FP64 parity bar ----

@pytest.mark.parametrize("N,eq", CASES_2D)
def test_float_float_contraction_2d(N, eq):
    p, s = make(2, N, (5, 3), eq, dtype="f64ff", epb=4, length=(1.0, 0.7, 1.0), velocity=(0.9, -0.6, 0))
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    check(p, s, U, dt, 2, 4, F64_TOL)


@pytest.mark.parametrize("dim,N,E,eq,rk", [(1, 3, (9,), 0, 4), (1, 6, (7,), 1, 6), (3, 2, (3, 2, 3), 1, 4),
                                           (3, 5, (2, 3, 2), 0, 3), (3, 3, (2, 2, 3), 1, 6), (2, 7, (4, 3), 1, 6),
                                           (3, 5, (3, 2, 3), 1, 3), (3, 5, (2, 3, 2), 1, 4), (3, 5, (2, 2, 3), 1, 6),
                                           (3, 7, (2, 2, 3), 1, 4), (3, 4, (2, 3, 2), 1, 4), (3, 6, (2, 2, 3), 1, 6),
                                           (3, 3, (3, 2, 2), 1, 3)])
def test_float_float_contraction_1d_3d_rk(dim, N, E, eq, rk):
    p, s = make(dim, N, E, eq, dtype="f64ff", epb=3, length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3))
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    check(p, s, U, dt, 3, rk, F64_TOL)
    if dim == 3 and eq == 1:
        # tiles of 1, 2, 4 (ragged) and 3 elements give the same bits
        outs = []
        for epb in (1, 2, 3, 4):
            _, t = make(dim, N, E, eq, dtype="f64ff", epb=epb, length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3))
            t.set_state(U)
            t.step(dt, 2, rk)
            outs.append(t.get_state())
            t.close()
        assert all(np.array_equal(o, outs[0]) for o in outs[1:])


def test_float_float_falls_back_to_fp64_for_unsplittable_values():
    """Advection is linear: a state of magnitude 1e-25 (below 2^-74, not splittable into normal
    floats) takes the FP64 contraction and still meets the FP64 bar; a state mixing tiny and
    ordinary values takes either path line by line."""
    p, s = make(2, 5, (6, 5), 0, dtype="f64ff", epb=4)
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    check(p, s, U * 1e-25, dt, 2, 4, F64_TOL)
    mixed = U.copy()
    mixed[:, ::2] *= 1e-25
    check(p, s, mixed, dt, 2, 4, F64_TOL)


def test_float_float_full_size_config2():
    p = orc.Problem(dim=2, degree=7, elems=(256, 256, 1), equation=0, flux=0, velocity=(1.0, 0.5, 0))
    X = orc.node_coords(p)
    U0 = inputs.gaussian_noise(X)
    dt = orc.stable_dt(p, U0, 0.1)
    ref = orc.step(p, U0, dt, 1, 4)
    s = Solver(2, 7, (256, 256), velocity=(1.0, 0.5, 0), dtype="f64ff")
    s.set_state(U0)
    s.step(dt, 1, 4)
    got = s.get_state()
    assert rel_l2(got, ref) < F64_TOL
    per_element_check(got, ref, F64_TOL)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64ff"])
@pytest.mark.parametrize("dim,N,E,vel", [(2, 5, (4, 5), (0.0, 0.7, 0.0)), (3, 3, (3, 2, 3), (0.5, 0.0, -0.3)),
                                         (3, 2, (2, 3, 2), (0.0, 0.0, 0.9)), (2, 7, (5, 4), (0.0, 0.7, 0.0)),
                                         (2, 3, (5, 4), (0.6, 0.0, 0.0)), (3, 5, (2, 3, 2), (0.5, 0.0, -0.3))])
def test_advection_with_zero_velocity_components(dim, N, E, vel, dtype):
    """An axis without velocity carries no flux: the kernel skips it (axis 0 included)."""
    p, s = make(dim, N, E, 0, dtype=dtype, epb=3, velocity=vel)
    U = initial(p)
    dt = orc.stable_dt(p, U, 0.2)
    if dtype == "f32":
        s.set_state(U)
        s.step(dt, 1, 4)
        assert rel_l2(s.get_state(), orc.step(p, U.astype(np.float32).astype(np.float64), dt, 1, 4)) < F32_TOL
    else:
        check(p, s, U, dt, 2, 4, F64_TOL)


# ---- the exact-mass variant (NDG_MASS_EXACT) against the oracle's exact-mass weak form ----

@pytest.mark.parametrize("dim,N,E,eq", [(1, 4, (7,), 1), (1, 3, (6,), 0), (2, 7, (5, 3), 0), (2, 7, (4, 3), 1),
                                        (2, 4, (5, 4), 1), (3, 2, (3, 2, 3), 1), (3, 5, (2, 3, 2), 1),
                                        (3, 3, (2, 2, 3), 0)])
def test_exact_mass_variant(dim, N, E, eq):
    """FP64 within 1e-12 per step (RK4 and RK6, both thread mappings, ragged tiles) and FP32 within
    its tolerance, on a state whose faces jump (the lift differs from the lumped one there)."""
    flux = 0 if eq == 0 else 1
    kw = dict(equation=eq, flux=flux, length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3), mass=nat.NDG_MASS_EXACT)
    p = orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - len(E)), equation=eq, flux=flux,
                    length=(1.0, 0.8, 1.2), velocity=(0.7, -0.4, 0.3), mass=orc.MASS_EXACT)
    U = initial(p)
    dt = 0.5 * orc.stable_dt(p, U, 0.2)
    for kern in (nat.NDG_KERNEL_LINE, nat.NDG_KERNEL_LINE_VAR):
        for rk in (4, 6):
            s = Solver(dim, N, E, elems_per_block=2, kernel=kern, **kw)
            check(p, s, U, dt, 2, rk, F64_TOL)
    s = Solver(dim, N, E, elems_per_block=3, dtype="f32", **kw)
    s.set_state(U)
    s.step(dt, 2, 4)
    ref = orc.step(p, U.astype(np.float32).astype(np.float64), dt, 2, 4)
    assert rel_l2(s.get_state(), ref) < 2 * F32_TOL
    # and it is a different scheme: the lumped solve moves away from it
    s = Solver(dim, N, E, elems_per_block=2, **dict(kw, mass=nat.NDG_MASS_LUMPED))
    s.set_state(U)
    s.step(dt, 2, 4)
    assert rel_l2(s.get_state(), orc.step(p, U, dt, 2, 4)) > 1e-9


def test_exact_mass_rejected_for_float_float_and_batches_apart():
    with pytest.raises(nat.NdgError) as ei:
        Solver(2, 3, (4, 4), dtype="f64ff", mass=nat.NDG_MASS_EXACT)
    assert ei.value.status == nat.NDG_EINVAL
    # a batch of an exact-mass and a lumped solve of the same shape: each as alone
    p = orc.Problem(dim=2, degree=5, elems=(4, 3, 1), equation=1, flux=1, mass=orc.MASS_EXACT)
    U = initial(p)
    dt = 0.5 * orc.stable_dt(p, U, 0.2)
    outs = []
    for m in (nat.NDG_MASS_EXACT, nat.NDG_MASS_LUMPED):
        s = Solver(2, 5, (4, 3), equation=1, mass=m)
        s.set_state(U)
        s.step(dt, 3, 4)
        outs.append(s.get_state())
    a = Solver(2, 5, (4, 3), equation=1, mass=nat.NDG_MASS_EXACT)
    b = Solver(2, 5, (4, 3), equation=1, mass=nat.NDG_MASS_LUMPED)
    a.set_state(U)
    b.set_state(U)
    batch = Batch([a, b])
    batch.step([dt, dt], 3, 4)
    assert np.array_equal(a.get_state(), outs[0]) and np.array_equal(b.get_state(), outs[1])
