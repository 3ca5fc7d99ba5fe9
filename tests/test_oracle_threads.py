"""The oracle's threaded split (orc_step_threads, the timed all-cores CPU baseline) and its
-O3 -march=native timing build against the checking build's single-threaded orc_step: bit for
bit, for every scheme, both equations, 1D/2D/3D, uneven element ranges (more threads than a
split into equal ranges allows, more threads than elements)."""
import numpy as np
import pytest

from oracle import oracle as orc
from tests.test_oracle_scheme import _prob, _random_state

ADV, EUL = orc.ADVECTION, orc.ISO_EULER

CASES = [(1, 3, (13,), ADV, 3), (2, 4, (5, 3), EUL, 4), (3, 2, (3, 2, 3), EUL, 6), (2, 7, (4, 5), ADV, 4),
         (3, 3, (2, 2, 3), ADV, 6), (1, 5, (7,), EUL, 3)]


@pytest.mark.parametrize("dim,N,E,eq,rk", CASES)
@pytest.mark.parametrize("threads", [1, 2, 5, 64])
def test_threaded_split_is_bitwise_the_single_thread_step(dim, N, E, eq, rk, threads):
    p = _prob(dim, N, E, eq=eq, length=(1.0, 0.7, 1.3))
    U = _random_state(p, 17)
    dt = 0.5 * orc.stable_dt(p, U, 0.1)
    ref = orc.step(p, U, dt, 3, rk)
    got = orc.step_threads(p, U, dt, 3, rk, threads=threads)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dim,N,E,eq,rk", CASES[:4])
def test_native_timing_build_is_bitwise_the_checking_build(dim, N, E, eq, rk):
    p = _prob(dim, N, E, eq=eq, length=(1.0, 0.7, 1.3))
    U = _random_state(p, 23)
    dt = 0.5 * orc.stable_dt(p, U, 0.1)
    ref = orc.step(p, U, dt, 2, rk)
    assert np.array_equal(orc.step_native(p, U, dt, 2, rk), ref)
    assert np.array_equal(orc.step_threads(p, U, dt, 2, rk, threads=3, native=True), ref)
