"""Multi-rank host logic of bench.py on CPU: two gloo ranks (no GPU needed).

The transforms shard only as independent replicas (one GPU per rank, no
exchange), so the only cross-rank logic is the barrier and the max/sum
reductions of the per-rank timings; these are checked here with world size 2.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_init("gloo")
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    mx = bench.max_over_ranks(10.0 + rank, w)
    sm = bench.sum_over_ranks(1.5 * (rank + 1), w)
    q.put((rank, mx, sm))
    dist.destroy_process_group()


def test_two_rank_reductions():
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
    assert [r[1] for r in res] == [11.0, 11.0]
    assert [r[2] for r in res] == [4.5, 4.5]


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.sum_over_ranks(3.25, 1) == 3.25
