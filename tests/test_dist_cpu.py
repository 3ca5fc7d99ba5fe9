"""The N > 1 path of bench.py on CPU: world-size-2 gloo process group, max-over-ranks timing and
the whole-job aggregation, and the reference arm running on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    class Args:
        impl = "reference"
    w, r, local, pg = bench.dist_setup(Args)
    assert (w, r) == (world, rank) and pg is not None
    # each rank "measured" a different time; everybody must see the maximum
    t = bench.max_over_ranks(pg, 10.0 + rank, None)
    bench.barrier(pg)
    # the whole-job value counts every rank's work over the slowest rank's time
    work_per_rank = 1000.0
    value = w * work_per_rank / t
    # the reference arm runs on rank 0 only
    ref_line = bench.run_reference(type("A", (), {"warmup": 0, "steps": 0})(), w, r) if r != 0 else "rank0"
    q.put((rank, t, value, ref_line))
    dist.destroy_process_group()


def test_two_rank_gloo_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [11.0, 11.0]
    assert all(abs(x[2] - 2 * 1000.0 / 11.0) < 1e-12 for x in res)
    assert res[1][3] is None  # rank 1 does no reference work
