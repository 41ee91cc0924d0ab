"""Write the oracle's converged cartograms of the named synthetic workloads to tests/golden/.

TEST INFRASTRUCTURE ONLY. This script calls the FP64 CPU oracle (oracle/) and the
seeded input generator (synth.py, loaded from its file so that nothing of the CUDA
library's binding is imported); it never touches the CUDA path. Each workload runs the
whole method -- rasterise, blurred forward transform, diffusion-flow integration with
adaptive predictor-corrector steps, vertex map, areas -- and repeats the integration
until the largest relative area error is below 1 % (main text, section on
benchmarking: the output of one integration is the input of the next; stopping
criterion on the relative area error).

Stored per workload (`<name>.npz`):
  map_sha256        SHA-256 of the generated input (values, ring offsets, ring regions,
                    vertices), so that a test can confirm it rebuilt the same map
  iterations, converged, status, steps_accepted, steps_rejected, max_area_error
  err               signed relative area error of every region after the last iteration
  vertex_index, xy  a fixed stride sample of the converged vertices
  cell_index, grid  projected position (X, Y) of a fixed sample of grid cells after every
                    outer iteration, [iterations, 2, n_cells]

Usage:  python oracle/make_golden.py [--out DIR] [workload ...]   (default: all of RUNS,
        written to tests/golden/)
The 1024^2 workload costs about 3000 attempted steps of O(L^3) direct sums: tens of
minutes on a few host cores.
"""
from __future__ import annotations

import hashlib
import importlib.util
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
GOLDEN = os.path.join(ROOT, "tests", "golden")

# outer-iteration budget large enough for every workload (the 512^2 clustered map
# needs about 190 iterations to resolve its smallest region)
RUNS = {
    "voronoi16_64": dict(max_iter=200, n_vertices=4096, n_cells=256),
    "clustered300_512": dict(max_iter=260, n_vertices=16384, n_cells=512),
    "powerlaw3000_1024": dict(max_iter=60, n_vertices=16384, n_cells=512),
    # the first frame of each of the two smaller grid sizes of the batched workload
    # (64 frames whose values drift by a multiplicative random walk)
    "batch_frame_128": dict(max_iter=200, n_vertices=8192, n_cells=256, batch_size=128),
    "batch_frame_256": dict(max_iter=200, n_vertices=8192, n_cells=256, batch_size=256),
}


def load_synth():
    spec = importlib.util.spec_from_file_location(
        "_golden_synth", os.path.join(ROOT, "paper_1802_07625_gb300", "synth.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


def map_sha256(m) -> str:
    h = hashlib.sha256()
    for a, dt in ((m.values, "<f8"), (m.ring_offsets, "<i8"), (m.ring_region, "<i4"), (m.xy, "<f8")):
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    return h.hexdigest()


def sample_indices(n: int, k: int) -> np.ndarray:
    """k distinct indices spread over [0, n): a fixed stride with a multiplicative offset."""
    if n <= k:
        return np.arange(n, dtype=np.int64)
    return (np.arange(k, dtype=np.int64) * n) // k


def batch_frame(synth, size: int):
    """(frame number, map) of the first frame of the batched workload with this grid size."""
    for f, m in enumerate(synth.make_batch()):
        if m.Lx == size:
            return f, m
    raise ValueError("no frame of size %d" % size)


def workload(synth, name: str):
    cfg = RUNS[name]
    if "batch_size" in cfg:
        f, m = batch_frame(synth, cfg["batch_size"])
        return m, float(synth.BATCH["blur"]), f
    m = synth.make_workload(name)
    return m, float(m.meta["blur"]), -1


def run(name: str, out_dir: str = GOLDEN) -> dict:
    sys.path.insert(0, ROOT)
    import oracle

    synth = load_synth()
    cfg = RUNS[name]
    m, blur, frame = workload(synth, name)
    t0 = time.time()
    res = oracle.cartogram(m, blur, keep_grids=True, max_iter=cfg["max_iter"])
    seconds = time.time() - t0
    vi = sample_indices(m.n_vertices, cfg["n_vertices"])
    ci = sample_indices(m.Lx * m.Ly, cfg["n_cells"])
    # the stride sample of cells lines up with rows; scatter it over the columns too
    ci = (ci * 7919) % (m.Lx * m.Ly)
    iy, ix = ci // m.Lx, ci % m.Lx
    grid = res.grids[:, :, iy, ix] if res.iterations else np.zeros((0, 2, ci.size))
    out = dict(map_sha256=map_sha256(m), iterations=res.iterations, converged=int(res.converged),
               status=res.status, steps_accepted=res.steps_accepted, steps_rejected=res.steps_rejected,
               max_area_error=res.max_area_error, blur=blur, max_iter=cfg["max_iter"], frame=frame,
               oracle_seconds=seconds, oracle_threads=oracle.num_threads())
    os.makedirs(out_dir, exist_ok=True)
    np.savez_compressed(os.path.join(out_dir, name + ".npz"), err=res.err, vertex_index=vi, xy=res.xy[vi],
                        cell_index=ci, grid=grid, meta=np.array(json.dumps(out)))
    return out


def main(argv):
    out_dir = GOLDEN
    if "--out" in argv:
        k = argv.index("--out")
        out_dir = argv[k + 1]
        argv = argv[:k] + argv[k + 2:]
    names = argv or list(RUNS)
    for name in names:
        info = run(name, out_dir)
        print(name, json.dumps(info), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
