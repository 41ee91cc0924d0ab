"""The multi-rank path of the benchmark (independent replicas, one per rank) on CPU with
the gloo backend and two ranks: the whole-job value is all ranks' updates over the
slowest rank's time, and the barrier/reductions work across processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench._dist()
    bench._barrier(w)
    # rank k did (k+1) * 1e9 updates in (k+2) seconds
    value = bench.replica_throughput(w, (r + 1) * 1e9, r + 2.0)
    q.put((r, w, value))
    dist.destroy_process_group()


def test_two_rank_replica_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, value in out:
        assert w == 2
        assert value == pytest.approx((1e9 + 2e9) / 3.0)
