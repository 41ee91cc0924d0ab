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


def _shard_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    from paper_1802_07625_gb300 import shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    frames = synth.make_batch(frames=10, sizes=(128, 256))
    costs = [shard.frame_cost(f.Lx, f.Ly) for f in frames]
    mine = shard.partition(costs, world)[rank]
    # each rank "runs" its frames: here the result is the frame's size and a rank tag
    res = shard.gather_results(world, rank, mine, [(frames[i].Lx, rank) for i in mine])
    # the re-split by measured step counts: every rank gathers every frame's count and
    # computes the same new split (here the "measured" steps are 10 * (frame index + 1))
    steps = shard.gather_results(world, rank, mine, [10 * (i + 1) for i in mine], all_ranks=True)
    parts = shard.partition(shard.measured_costs([(f.Lx, f.Ly) for f in frames], steps), world)
    q.put((rank, mine, res, steps, parts))
    dist.destroy_process_group()


def test_two_rank_batch_sharding_gathers_every_frame_once():
    from paper_1802_07625_gb300 import shard, synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    frames = synth.make_batch(frames=10, sizes=(128, 256))
    (r0, mine0, res0, steps0, parts0), (r1, mine1, res1, steps1, parts1) = out
    assert steps0 == steps1 == [10 * (i + 1) for i in range(10)]
    assert parts0 == parts1 and sorted(parts0[0] + parts0[1]) == list(range(10))
    assert sorted(mine0 + mine1) == list(range(10)) and not set(mine0) & set(mine1)
    assert res1 is None
    assert [r[0] for r in res0] == [f.Lx for f in frames]
    assert all(res0[i][1] == 0 for i in mine0) and all(res0[i][1] == 1 for i in mine1)
