"""The split of a batch's frames between ranks (host logic, no GPU): every frame on
exactly one rank, the same split on every rank, and the greedy longest-first bound
(makespan at most the mean load plus the largest frame)."""
import numpy as np
import pytest

from paper_1802_07625_gb300 import shard, synth


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8, 100])
def test_partition_covers_every_frame_once_and_balances(world):
    rng = np.random.default_rng(world)
    costs = [shard.frame_cost(L, L) for L in rng.choice([128, 256, 512, 1024], 64)]
    parts = shard.partition(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(64))
    assert parts == shard.partition(list(costs), world)  # deterministic
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) <= sum(costs) / world + max(costs) + 1e-6
    if world >= 64:
        assert all(len(p) <= 1 for p in parts)


def test_partition_of_equal_costs_is_round_robin_sized():
    parts = shard.partition([1.0] * 10, 4)
    assert sorted(len(p) for p in parts) == [2, 2, 3, 3]


def test_partition_of_the_batched_workload():
    frames = synth.make_batch()
    costs = [shard.frame_cost(f.Lx, f.Ly) for f in frames]
    for world, slack in ((2, 1.01), (4, 1.03)):
        loads = [sum(costs[i] for i in p) for p in shard.partition(costs, world)]
        assert max(loads) <= slack * sum(costs) / world
    # on 8 ranks the 17 frames of 1024^2 (41 % of a rank's mean load each) cannot split
    # evenly: three ranks hold three of them, which is the optimum for those frames
    big = max(costs)
    loads = [sum(costs[i] for i in p) for p in shard.partition(costs, 8)]
    assert max(loads) <= 3 * big + 1e-6 + sum(costs[i] for i in range(64) if costs[i] < big) / 8


def test_partition_and_gather_reject_bad_input():
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)
    with pytest.raises(ValueError):
        shard.partition([1.0, float("nan")], 2)
    with pytest.raises(ValueError):
        shard.gather_results(1, 0, [0, 1], [None])
    assert shard.gather_results(1, 0, [1, 0], ["b", "a"]) == ["a", "b"]


def test_measured_costs_fill_gaps_from_frames_of_the_same_size():
    sizes = [(128, 128), (256, 256), (128, 128), (256, 256), (512, 512)]
    steps = [100, None, None, 40, None]
    c = shard.measured_costs(sizes, steps)
    assert c[0] == 128 * 128 * 100
    assert c[1] == 256 * 256 * 40      # the nearest later frame of its size
    assert c[2] == 128 * 128 * 100     # the nearest earlier frame of its size
    assert c[3] == 256 * 256 * 40
    assert c[4] == shard.frame_cost(512, 512)  # no measurement of that size: the size model
    with pytest.raises(ValueError):
        shard.measured_costs(sizes, steps[:2])


def test_measured_costs_balance_better_than_the_size_model():
    # frames of one size whose step counts differ by 20x: the size model sees equal costs,
    # the measured costs let the split balance the real work
    rng = np.random.default_rng(3)
    sizes = [(256, 256)] * 16
    steps = list(rng.integers(50, 1000, 16))
    real = [256 * 256 * s for s in steps]
    by_size = shard.partition([shard.frame_cost(*sz) for sz in sizes], 4)
    by_steps = shard.partition(shard.measured_costs(sizes, steps), 4)

    def makespan(parts):
        return max(sum(real[i] for i in p) for p in parts)

    assert makespan(by_steps) <= makespan(by_size)
    assert makespan(by_steps) <= sum(real) / 4 + max(real)
