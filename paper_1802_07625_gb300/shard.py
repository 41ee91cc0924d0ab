"""Sharding a batch of independent cartograms across ranks (one process per GPU).

The frames of a batch share nothing: each is a whole cartogram of its own map, so the
ranks split the frames between them and run their shares as independent batches, with
no collective on the data path. The only exchange is the gather of the per-frame
results to rank 0 on the host at the end.

The split is a greedy longest-first balance (each frame, costliest first, goes to the
rank with the least work so far; ties to the lower rank), which gives a makespan within
4/3 of the optimum. A frame's cost is its grid-point updates to convergence,
Lx * Ly * (attempted steps). Before any run the attempted steps are unknown, and the size
model takes them proportional to the grid's larger side (the step size is capped at one
cell of displacement per step and the displacements, in cells, grow with the grid). That
model can be off by an order of magnitude: frames of one size need from a few to over a
hundred outer iterations. Once a run has measured each frame's attempted steps, the split
uses those (measured_costs); frames drift slowly, so a frame without a measurement takes
the steps of the nearest earlier measured frame of its size.
"""


def frame_cost(Lx, Ly, steps=None):
    """Expected grid-point updates of one frame: Lx * Ly * steps, with steps taken as
    max(Lx, Ly) when not given."""
    return float(Lx) * float(Ly) * float(max(Lx, Ly) if steps is None else steps)


def measured_costs(sizes, steps):
    """Costs Lx * Ly * steps from measured attempted steps. `sizes` lists (Lx, Ly) per
    frame and `steps` the measured attempted steps per frame (None where not measured):
    such a frame takes the steps of the nearest earlier measured frame of the same size,
    else the nearest later one, else the size model."""
    if len(sizes) != len(steps):
        raise ValueError("one step count per frame")
    out = []
    for i, (lx, ly) in enumerate(sizes):
        st = steps[i]
        if st is None:
            same = [k for k in range(len(sizes)) if tuple(sizes[k]) == (lx, ly) and steps[k] is not None]
            earlier = [k for k in same if k < i]
            later = [k for k in same if k > i]
            st = steps[earlier[-1]] if earlier else (steps[later[0]] if later else None)
        if st is not None and not (st >= 0):
            raise ValueError("step counts must be non-negative")
        out.append(frame_cost(lx, ly, st))
    return out


def partition(costs, world):
    """Split frame indices 0..len(costs)-1 over `world` ranks: a list of `world` sorted
    index lists, each frame in exactly one. Deterministic, so every rank computes the same
    split without communicating."""
    if world < 1:
        raise ValueError("world must be at least 1")
    if any(not (c >= 0.0) for c in costs):
        raise ValueError("frame costs must be non-negative numbers")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_results(world, rank, frames, results, all_ranks=False):
    """Collect each rank's per-frame results on rank 0 (on every rank with all_ranks), in
    frame order: returns the list indexed by frame there and None elsewhere. `frames` are
    this rank's frame indices and `results` its results for them (any picklable objects),
    in the same order."""
    if len(frames) != len(results):
        raise ValueError("one result per frame")
    if world == 1:
        out = [None] * len(frames)
        for i, r in zip(frames, results):
            out[i] = r
        return out
    import torch.distributed as dist
    got = [None] * world
    dist.all_gather_object(got, (list(frames), list(results)))
    if rank != 0 and not all_ranks:
        return None
    n = sum(len(f) for f, _ in got)
    out = [None] * n
    seen = set()
    for f, res in got:
        for i, r in zip(f, res):
            if i in seen or not 0 <= i < n:
                raise RuntimeError("frame %d gathered twice or out of range" % i)
            seen.add(i)
            out[i] = r
    return out
