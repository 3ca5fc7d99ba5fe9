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
    U[0] = 1.0 + 0.1 * np.sin(2 * np.pi * X[0]) * np.cos(2 * np.pi * X[1])
    for a in range(1, p.nvar):
        U[a] = 0.2 * np.cos(2 * np.pi * (X[0] + seed * X[1]) + a)
    return U


def _compare(got, want):
    """The tolerances of the norms parity test."""
    assert abs(got[0] - want.l2) < 1e-13 * max(1.0, want.l2)
    assert abs(got[1] - want.linf) < 1e-15 * max(1.0, want.linf)
    np.testing.assert_allclose(got[2:2 + 4], list(want.integral), rtol=1e-13, atol=1e-14)
    assert abs(got[6] - want.max_speed) < 1e-13 * max(1.0, want.max_speed)
    assert int(got[7]) == want.nonfinite


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_norms_match_the_allocating_entry_point_twice_in_a_row(dtype):
    p = orc.Problem(dim=2, degree=5, elems=(7, 6, 1), equation=1, flux=1)
    s = Solver(2, 5, (7, 6), equation=1, dtype=dtype)
    tdt = s.torch_dtype
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    # first call: norms of U - ref; second call: norms of another state, no reference and fewer
    # blocks, so stale partial sums of the first call would show up if they leaked
    cases = [(_state(p, 1), _state(p, 2), 0), (_state(p, 3), None, 37)]
    for U, ref, nblocks in cases:
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


def test_noalloc_rejects_too_many_blocks():
    cfg = nat.ndg_config_init()
    u = torch.zeros(cfg.elems[0] * cfg.elems[1] * 64, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(nat.NdgError) as ei:
        nat.ndg_norms_noalloc(cfg, u.data_ptr(), None, 1025, out.data_ptr(), 0)
    assert ei.value.status == nat.NDG_EINVAL and "1024" in str(ei.value)
