"""ndg_norms_noalloc: norms for callers that may not allocate device memory.

Some applications give all of a GPU's memory to their own pool allocator when they start (or
share the device under a fixed memory split), so a library that calls cudaMalloc behind their back
fails or corrupts their accounting; others run latency-critical loops where the device-wide
synchronisation cudaMalloc/cudaFree can cause is not acceptable.  For them the library offers one
norms entry point that keeps its per-block partial sums in a fixed array compiled into the
library and takes every input and output from the caller.

This file is collected last on purpose (its name sorts after the other test files), so a run that
stops at the first failure has already run everything else.  It must also pass alone in a fresh
process."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05254_b300 import native as nat  # noqa: E402
from paper_2510_05254_b300.solver import Solver  # noqa: E402


def _state(p, seed):
    X = orc.node_coords(p)
    U = np.zeros(p.shape)
    U[0] = 1.0 + 0.1 * np.sin(2 * np.pi * X[0]) * np.cos(2 * np.pi * X[-1])
    for a in range(1, p.nvar):
        U[a] = 0.2 * np.cos(2 * np.pi * (X[0] + seed * X[-1]) + a)
    if p.equation == 0:
        U[0] += 0.3 * np.sin(2 * np.pi * seed * X[-1])
    return U


def _compare(got, want):
    """The tolerances of the norms parity test."""
    assert abs(got[0] - want.l2) < 1e-13 * max(1.0, want.l2)
    assert abs(got[1] - want.linf) < 1e-15 * max(1.0, want.linf)
    np.testing.assert_allclose(got[2:2 + 4], list(want.integral), rtol=1e-13, atol=1e-14)
    assert abs(got[6] - want.max_speed) < 1e-13 * max(1.0, want.max_speed)
    assert int(got[7]) == want.nonfinite


CASES = [(1, 4, (9,)), (2, 5, (7, 6)), (3, 3, (3, 4, 2))]


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64ff"])
@pytest.mark.parametrize("eq", [0, 1])
@pytest.mark.parametrize("dim,N,E", CASES)
def test_noalloc_norms_match_the_allocating_entry_point_twice_in_a_row(dim, N, E, eq, dtype):
    """Advection (max speed = sum |a|) and isothermal Euler, 1D/2D/3D, every precision: two calls
    in a row, the second with another state, no reference and fewer blocks."""
    p = orc.Problem(dim=dim, degree=N, elems=E + (1,) * (3 - dim), equation=eq, flux=1 if eq else 0,
                    velocity=(0.7, -0.4, 0.3))
    s = Solver(dim, N, E, equation=eq, dtype=dtype, velocity=(0.7, -0.4, 0.3))
    tdt = s.torch_dtype
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    for U, ref, nblocks in [(_state(p, 1), _state(p, 2), 0), (_state(p, 3), None, 37)]:
        u_dev = torch.tensor(U, dtype=tdt, device="cuda")
        r_dev = torch.tensor(ref, dtype=tdt, device="cuda") if ref is not None else None
        s.set_state(u_dev)
        want = nat.ndg_norms(s.ctx, r_dev.data_ptr() if r_dev is not None else None, True)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream().cuda_stream
        nat.ndg_norms_noalloc(s.cfg, u_dev.data_ptr(), r_dev.data_ptr() if r_dev is not None else None,
                              nblocks, out.data_ptr(), stream)
        torch.cuda.synchronize()
        _compare(out.cpu().numpy(), want)
    s.close()


def test_noalloc_counts_nonfinite_values_and_ignores_stale_partials():
    """NaN / inf values are counted in out[7].  A call over an all-NaN state large enough that
    each of its 1024 blocks has nodes to reduce leaves NaN in every partial-sum slot of the shared
    scratch; a later call with fewer blocks reads only the partials it wrote itself, so its result
    is unaffected."""
    p = orc.Problem(dim=2, degree=5, elems=(7, 6, 1), equation=1, flux=1)
    s = Solver(2, 5, (7, 6), equation=1, dtype="f64")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    bad = _state(p, 1)
    bad[0, 3, 7], bad[2, 40, 0], bad[1, 0, 0] = np.nan, np.inf, -np.inf
    b_dev = torch.tensor(bad, device="cuda")
    nat.ndg_norms_noalloc(s.cfg, b_dev.data_ptr(), None, 0, out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert int(out[7].item()) == 3
    # 64 x 64 elements of degree 7: 262144 nodes, one per thread of the 1024 x 256 reduction
    big = Solver(2, 7, (64, 64), equation=1, dtype="f64")
    nan_dev = torch.full((3, 64 * 64, 64), float("nan"), dtype=torch.float64, device="cuda")
    nat.ndg_norms_noalloc(big.cfg, nan_dev.data_ptr(), None, 1024, out.data_ptr(), stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert int(got[7]) == 3 * 64 * 64 * 64 and np.isnan(got[0])
    big.close()
    good = _state(p, 2)
    g_dev = torch.tensor(good, device="cuda")
    s.set_state(g_dev)
    want = nat.ndg_norms(s.ctx)
    torch.cuda.synchronize()
    nat.ndg_norms_noalloc(s.cfg, g_dev.data_ptr(), None, 5, out.data_ptr(), stream)
    torch.cuda.synchronize()
    _compare(out.cpu().numpy(), want)
    s.close()


def test_noalloc_rejects_too_many_blocks():
    cfg = nat.ndg_config_init()
    u = torch.zeros(cfg.elems[0] * cfg.elems[1] * 64, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(nat.NdgError) as ei:
        nat.ndg_norms_noalloc(cfg, u.data_ptr(), None, 1025, out.data_ptr(), 0)
    assert ei.value.status == nat.NDG_EINVAL and "1024" in str(ei.value)
