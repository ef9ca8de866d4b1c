"""The replica path's host logic on two CPU ranks (gloo): every stream goes
to exactly one rank, the job time is the slowest rank's, and the job's
bytes are the sum over ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = bench.shard_range(8193, rank, world)
    t = bench.reduce_max(10.0 * (rank + 1), dist, "cpu")
    b = bench.reduce_sum(float(hi - lo), dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, lo, hi, t, b))


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spans = [(lo, hi) for _, lo, hi, _, _ in res]
    assert spans[0][0] == 0 and spans[-1][1] == 8193
    assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
    assert all(t == 10.0 * world for *_, t, _ in res)
    assert all(b == 8193.0 for *_, b in res)          # every stream counted once
