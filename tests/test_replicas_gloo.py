"""The N > 1 path of the benchmark on CPU: world-size-2 gloo ranks.

The step does not shard (each GPU runs a whole, independent domain), so the only
multi-rank logic is the barrier around the timed region, the max over ranks of
its duration, and the whole-job throughput; the reference arm runs on rank 0
only.  These run here as two spawned gloo processes on 127.0.0.1.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    rep = bench.Replicas("gloo")
    rep.barrier()
    elapsed = 1.0 + rank  # rank 1 is the slowest
    m = rep.max(elapsed)
    value = bench.aggregate_mlups(1000, 10, rep.world, m)
    ref_rc = None
    if rank == 1:
        class A:
            steps, warmup = 1, 3
        ref_rc = bench.run_reference(A)  # non-zero ranks exit 0 without work
    rep.close()
    q.put((rank, m, value, ref_rc))


def test_two_gloo_replicas():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, value, ref_rc in res:
        assert m == 2.0                                  # max over ranks
        assert abs(value - 2 * 1000 * 10 / 2.0 / 1e6) < 1e-15  # all ranks' updates / slowest time
    assert res[1][3] == 0
