"""The stored oracle results in tests/golden/ against the committed oracle (no GPU).

Each file is written by oracle/make_golden.py. The 64^2 workload is cheap enough to
rerun here: the committed oracle must reproduce its stored converged cartogram, so the
fixtures cannot drift from the oracle's arithmetic unnoticed. For the larger workloads
only the file's structure and the seeded input are checked (their oracle runs take
minutes to tens of minutes)."""
import os

import numpy as np
import pytest

from paper_1802_07625_gb300 import synth
from test_gpu_golden import GOLDEN, golden_map, load_golden

NAMES = ["voronoi16_64", "clustered300_512", "powerlaw3000_1024", "batch_frame_128", "batch_frame_256"]


def test_small_fixture_is_reproduced_by_the_oracle(orc):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(
        os.path.dirname(GOLDEN), "..", "oracle", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    g = load_golden("voronoi16_64")
    m = golden_map("voronoi16_64", g["meta"])
    res = orc.cartogram(m, g["meta"]["blur"], keep_grids=True, max_iter=g["meta"]["max_iter"])
    assert (res.iterations, res.steps_accepted, res.steps_rejected) == \
        (g["meta"]["iterations"], g["meta"]["steps_accepted"], g["meta"]["steps_rejected"])
    # the oracle's rasteriser adds the rings' coverages in a thread-dependent order, so
    # reruns differ by rounding (~1e-13 grid units after the 11 iterations of this map)
    assert np.max(np.abs(res.xy[g["vertex_index"]] - g["xy"])) < 1e-11
    assert np.max(np.abs(res.err - g["err"])) < 1e-11
    ci = g["cell_index"]
    got = res.grids[:, :, ci // m.Lx, ci % m.Lx]
    assert np.max(np.abs(got - g["grid"])) < 1e-11
    # the sampled indices are what the script's rule gives
    assert np.array_equal(g["vertex_index"], mg.sample_indices(m.n_vertices, mg.RUNS["voronoi16_64"]["n_vertices"]))


@pytest.mark.parametrize("name", NAMES)
def test_fixture_structure(name):
    g = load_golden(name)
    meta = g["meta"]
    m = golden_map(name, meta)  # rebuilds the seeded map and checks its hash
    K = meta["iterations"]
    assert meta["converged"] == 1 and meta["status"] == 0 and meta["max_area_error"] < 0.01
    assert g["grid"].shape == (K, 2, g["cell_index"].size)
    assert g["err"].shape == (m.n_regions,) and np.max(np.abs(g["err"])) == pytest.approx(meta["max_area_error"])
    assert g["xy"].shape == (g["vertex_index"].size, 2)
    assert np.all(g["grid"] >= 0) and np.all(g["grid"][:, 0] <= m.Lx) and np.all(g["grid"][:, 1] <= m.Ly)
