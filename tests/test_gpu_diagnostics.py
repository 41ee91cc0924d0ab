"""Diagnostics of the composed projection on the GPU against the oracle, through the
C-ABI: the Tissot angular-distortion measures (SI section 3) and the inverse map (the
main text's inverse graticule). Both sides work in FP64 on the same grids (the GPU's
history, read back), so they agree to rounding: 1e-9."""
import numpy as np
import pytest

import paper_1802_07625_gb300 as P
from paper_1802_07625_gb300 import synth

pytestmark = pytest.mark.gpu


def _grids(c, m):
    """The context's history as projected positions [K][2][Ly][Lx] (oracle layout)."""
    xc = np.arange(m.Lx) + 0.5
    yc = np.arange(m.Ly) + 0.5
    out = []
    for k in range(c.history_length()):
        g = c.grid(k)
        out.append(np.stack([g[..., 0], g[..., 1]]))
    return np.array(out) if out else np.zeros((0, 2, m.Ly, m.Lx))


@pytest.mark.parametrize("precision,L", [("fp64", 64), ("mixed", 64), ("mixed", 128)])
def test_distortion_and_inverse_match_oracle(orc, precision, L):
    m = synth.make_workload("voronoi16_64", L=L, n=16 if L == 64 else 40)
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision=precision) as c:
        c.set_map(m)
        assert c.distortion() == {"e_a": 0.0, "e_inf": 0.0, "et_a": 0.0, "et_inf": 0.0}  # identity
        c.integrate()
        d = c.distortion()
        g = _grids(c, m)
        rng = np.random.default_rng(21)
        q = np.concatenate([rng.uniform(0.0, L, (2000, 2)), [[0.05, 0.1], [L - 0.05, 0.2], [0.3, L - 0.01]]])
        back = c.inverse_project(q)
        fwd = c.project(back)
    ref = orc.distortion(g)
    got = np.array([d["e_a"], d["e_inf"], d["et_a"], d["et_inf"]])
    assert np.all(np.abs(got - ref) <= 1e-9 * np.maximum(1.0, np.abs(ref)))
    assert ref[1] > 0.05
    # preimages agree with the oracle's (an exhaustive search over the quads), and the
    # forward map sends them back onto the query points
    # (the bilinear extension across the wall bands need not cover the box exactly, so a
    # query point very close to the box edge may have no preimage: NaN on both sides)
    ref_inv = orc.inverse_points(g, q)
    ok = ~np.isnan(ref_inv[:, 0])
    assert ok.mean() > 0.99
    assert np.array_equal(ok, ~np.isnan(back[:, 0]))
    assert np.max(np.abs(back[ok] - ref_inv[ok])) < 1e-9
    assert np.max(np.abs(fwd[ok] - q[ok])) < 1e-9


def test_inverse_of_projected_points_round_trips():
    m = synth.make_workload("voronoi16_64")
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="mixed") as c:
        c.set_map(m)
        c.integrate()
        back = c.inverse_project(c.vertices())
        # points outside the box have no preimage
        out = c.inverse_project(np.array([[-3.0, 10.0], [10.0, 70.0]]))
    assert np.max(np.abs(back - m.xy)) < 1e-9
    assert np.all(np.isnan(out))


@pytest.mark.slow
def test_diagnostics_at_1024(orc):
    m = synth.make_workload("powerlaw3000_1024")
    blur = synth.WORKLOADS["powerlaw3000_1024"]["blur"]
    with P.Cartogram(m.Lx, m.Ly, blur, precision="mixed", max_iter=100) as c:
        c.set_map(m)
        c.integrate()
        d = c.distortion()
        g = _grids(c, m)
        rng = np.random.default_rng(22)
        p = rng.uniform(0.0, m.Lx, (20000, 2))
        q = c.project(p)
        back = c.inverse_project(q)
    ref = orc.distortion(g)
    got = np.array([d["e_a"], d["e_inf"], d["et_a"], d["et_inf"]])
    # e_inf is infinite where the first integration folded quads (det J = 0 or < 0 gives
    # s2 -> 0): compare the finite measures, and that both sides see the fold
    assert np.all(np.abs(got[[0, 2, 3]] - ref[[0, 2, 3]]) <= 1e-9 * np.maximum(1.0, np.abs(ref[[0, 2, 3]])))
    assert got[1] == ref[1] or abs(got[1] - ref[1]) <= 1e-9 * abs(ref[1])
    # the first integration folds ~1e-4 of the quads: a point whose image lies where the
    # map folded has more than one preimage; all others come back
    err = np.max(np.abs(back - p), axis=1)
    assert np.mean(err < 1e-9) > 0.999


@pytest.mark.parametrize("name,precision", [("voronoi16_64", "fp64"), ("holes", "fp64"),
                                            ("clustered300_512", "mixed"), ("powerlaw3000_1024", "mixed")])
def test_polygon_measures_match_oracle(name, precision):
    # SI section 4: mean aspect ratio of the minimum-area bounding rectangles, and the
    # relative position error of the centroids, against the oracle on the GPU's vertices.
    # The hulls may differ in points collinear to within rounding (the GPU's orientation
    # test treats 1e-12 relative as collinear), which moves the extents by ~1e-12: alpha
    # to 1e-10
    from oracle import polygon as pg
    m = synth.holes_map(64) if name == "holes" else synth.make_workload(name)
    blur = synth.WORKLOADS[name]["blur"] if name in synth.WORKLOADS else 1.0
    with P.Cartogram(m.Lx, m.Ly, blur, precision=precision) as c:
        c.set_map(m)
        pm0 = c.polygon_measures()
        c.integrate()
        pm = c.polygon_measures()
        xy = c.vertices()
    args = (m.n_regions, m.ring_offsets, m.ring_region)
    a_in = pg.mean_aspect_ratio(*args, m.xy)
    a_out = pg.mean_aspect_ratio(*args, xy)
    theta = pg.relative_position_error(pg.region_centroids(*args, m.xy), pg.region_centroids(*args, xy))
    assert pm0["theta"] == 0.0 and pm0["alpha"] == pm0["alpha_input"]
    assert abs(pm0["alpha"] - a_in) <= 1e-10 * a_in
    assert abs(pm["alpha_input"] - a_in) <= 1e-10 * a_in
    assert abs(pm["alpha"] - a_out) <= 1e-10 * a_out
    # theta sums p (p - 1) / 2 angles (4.5 million at 1024^2) in a different order on each
    # side: 1e-10
    assert abs(pm["theta"] - theta) <= 1e-10 * max(theta, 1e-3)
    assert 0.0 < pm["theta"] < 0.5 and pm["alpha"] >= 1.0
