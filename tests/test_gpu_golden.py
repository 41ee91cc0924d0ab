"""Converged cartograms of the named workloads against the FP64 oracle's stored results.

tests/golden/<name>.npz is written by oracle/make_golden.py, which runs the oracle alone
(the whole method, repeated until the largest relative area error is below 1 %: main
text, section on benchmarking). Here the library runs the same workload through the C-ABI
in both precisions and is compared with that file:
  - the rebuilt input map must be byte-identical to the one the oracle ran;
  - FP64 path: the same number of outer iterations and of accepted / rejected steps,
    every sampled vertex and projected grid point of every iteration within 1e-9 grid
    units, area errors within 1e-9;
  - mixed paths (FP32 transforms, and FP32 pass 1 with pass 2 in float-float): the same
    number of outer iterations, sampled vertices within 1e-3 grid units, area errors within
    1e-4.
The 512^2 and 1024^2 workloads are the full configurations of the benchmark.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import paper_1802_07625_gb300 as P
from paper_1802_07625_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

FP64_TOL = 1e-9     # grid units: FP64 path against the FP64 oracle
MIXED_TOL = 1e-3    # grid units: mixed path against the FP64 oracle
AREA_TOL = 1e-4     # relative area errors, mixed path


def _sha(m):
    h = hashlib.sha256()
    for a, dt in ((m.values, "<f8"), (m.ring_offsets, "<i8"), (m.ring_region, "<i4"), (m.xy, "<f8")):
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    return h.hexdigest()


def load_golden(name):
    path = os.path.join(GOLDEN, name + ".npz")
    if not os.path.exists(path):
        pytest.skip("no stored oracle result %s (oracle/make_golden.py)" % name)
    z = np.load(path)
    g = {k: z[k] for k in z.files if k != "meta"}
    g["meta"] = json.loads(str(z["meta"]))
    return g


def golden_map(name, meta):
    if name.startswith("batch_frame_"):
        m = synth.make_batch()[meta["frame"]]
    else:
        m = synth.make_workload(name)
    assert _sha(m) == meta["map_sha256"], "the seeded input map differs from the one the oracle ran"
    return m


def _run(m, blur, precision):
    with P.Cartogram(m.Lx, m.Ly, blur, precision=precision) as c:
        c.set_map(m)
        st = c.integrate()
        xy = c.vertices()
        err = c.area_errors()
        grids = [c.grid(k) for k in range(c.history_length())]
    return st, xy, err, grids


def check_fp64(name, g, st, xy, err, grids):
    meta = g["meta"]
    assert st.converged and meta["converged"]
    assert (st.iterations, st.steps_accepted, st.steps_rejected) == \
        (meta["iterations"], meta["steps_accepted"], meta["steps_rejected"]), name
    d = np.max(np.abs(xy[g["vertex_index"]] - g["xy"]))
    assert d < FP64_TOL, (name, d)
    assert np.max(np.abs(err - g["err"])) < FP64_TOL, name
    ci = g["cell_index"]
    for k, grid in enumerate(grids):
        got = grid.reshape(-1, 2)[ci].T  # (X, Y) of the sampled cells
        assert np.max(np.abs(got - g["grid"][k])) < FP64_TOL, (name, k)


def check_mixed(name, g, st, xy, err):
    meta = g["meta"]
    assert st.converged
    assert st.iterations == meta["iterations"], (name, st.iterations, meta["iterations"])
    d = np.max(np.abs(xy[g["vertex_index"]] - g["xy"]))
    assert d < MIXED_TOL, (name, d)
    assert np.max(np.abs(err - g["err"])) < AREA_TOL, name
    assert st.max_area_error < 0.01


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["voronoi16_64", "clustered300_512", "powerlaw3000_1024"])
def test_converged_cartogram_matches_stored_oracle(name):
    g = load_golden(name)
    m = golden_map(name, g["meta"])
    blur = g["meta"]["blur"]
    st, xy, err, grids = _run(m, blur, "fp64")
    check_fp64(name, g, st, xy, err, grids)
    for precision in ("mixed", "mixed_ff"):
        st, xy, err, _ = _run(m, blur, precision)
        check_mixed(name, g, st, xy, err)
