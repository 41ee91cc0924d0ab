"""GPU path vs the FP64 CPU oracle, element by element, through the C-ABI.

Tolerances:
  FP64 path   1e-9 grid units on positions (the accuracy target of the method's
              FP64 implementation); fields 1e-10 relative to their scale.
  mixed path  1e-3 grid units on positions; fields 2e-5 relative (FP32 transforms
              of length <= 1024 accumulate ~log2(N) roundings of 6e-8).
  areas       relative area errors within 1e-4 of the oracle's.
Step counts must agree exactly: both sides take the accept/reject decisions in FP64
(FP64 path), and a decision flip would show up as a count difference.
"""
import math

import numpy as np
import pytest

import paper_1802_07625_gb300 as P
from paper_1802_07625_gb300 import synth

pytestmark = pytest.mark.gpu

FP64_POS_TOL = 1e-9
MIXED_POS_TOL = 1e-3
AREA_TOL = 1e-4


def _oracle_density(orc, m):
    A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, m.xy)
    rho = orc.rasterize(m.Lx, m.Ly, m.values, A, m.ring_offsets, m.ring_region, m.xy)
    return rho / (m.values.sum() / A.sum())


def _small_map(L=64, n=16, name="voronoi16_64"):
    return synth.make_workload(name, L=L, n=n)


def _ctx(m, blur, precision, **kw):
    c = P.Cartogram(m.Lx, m.Ly, blur, precision=precision, **kw)
    c.set_map(m)
    return c


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("L", [64, 128])
def test_density_matches_oracle(orc, precision, L):
    m = _small_map(L=L, n=16 if L == 64 else 40)
    with _ctx(m, 1.0, precision) as c:
        got = c.density()
    ref = _oracle_density(orc, m)
    # exact coverage by two different algorithms (edge accumulation vs polygon clipping)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-11)])
@pytest.mark.parametrize("shape", [(64, 64), (32, 64), (64, 16), (8, 8)])
def test_spectrum_matches_oracle(orc, precision, tol, shape):
    Ly, Lx = shape
    ring = synth.rectangle_ring(0.3 * Lx, 0.2 * Ly, 0.71 * Lx, 0.9 * Ly, 0.7)
    one = synth.RegionMap(Lx, Ly, np.array([2.0]), np.array([0, len(ring)]),
                          np.array([0], dtype=np.int32), ring)
    strips = synth.strip_map(Lx, Ly, [0, Lx // 4, Lx // 2, Lx], [1.0, 3.0, 0.5], spacing=0.6)
    for mm in (one, strips):
        with _ctx(mm, 1.3, precision) as c:
            got = c.spectrum()
        ref = orc.forward(_oracle_density(orc, mm), 1.3)
        assert np.max(np.abs(got - ref)) < tol * np.max(np.abs(ref))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 2e-5), ("mixed_ff", 2e-5)])
@pytest.mark.parametrize("shape", [(64, 64), (16, 64), (128, 32)])
@pytest.mark.parametrize("t", [0.0, 0.7, 25.0])
def test_velocity_matches_oracle(orc, precision, tol, shape, t):
    Ly, Lx = shape
    m = synth.strip_map(Lx, Ly, [0, Lx // 4, Lx // 2, Lx], [1.0, 3.0, 0.5], spacing=0.6) \
        if Lx != Ly else _small_map(L=Lx)
    with _ctx(m, 1.0, precision) as c:
        c.spectrum()
        rho, v = c.velocity(t)
    spec = orc.forward(_oracle_density(orc, m), 1.0)
    r0, gx, gy = orc.fields(spec, t)
    vx, vy, _ = orc.velocity(r0, gx, gy)
    assert np.max(np.abs(rho - r0)) < tol * np.max(np.abs(r0))
    scale = max(np.max(np.hypot(vx, vy)), 1e-30)
    assert np.max(np.abs(v[..., 0] - vx)) < tol * scale * 4
    assert np.max(np.abs(v[..., 1] - vy)) < tol * scale * 4


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5), ("mixed_ff", 1e-5)])
def test_heun_step_matches_oracle(orc, precision, tol):
    m = _small_map()
    Lx, Ly = m.Lx, m.Ly
    rng = np.random.default_rng(5)
    disp = rng.uniform(-3, 3, (Ly, Lx, 2))
    # keep every point inside the box, some on and near the walls
    xc = np.arange(Lx)[None, :] + 0.5
    yc = np.arange(Ly)[:, None] + 0.5
    disp[..., 0] = np.clip(xc + disp[..., 0], 0, Lx) - xc
    disp[..., 1] = np.clip(yc + disp[..., 1], 0, Ly) - yc
    t, h = 0.3, 0.45
    with _ctx(m, 1.0, precision) as c:
        c.spectrum()
        out, err = c.heun_step(t, h, disp)
    spec = orc.forward(_oracle_density(orc, m), 1.0)
    v0 = orc.velocity(*orc.fields(spec, t))
    v1 = orc.velocity(*orc.fields(spec, t + h))
    x = (xc + disp[..., 0]).ravel()
    y = (yc + disp[..., 1]).ravel()
    _, _, xcor, ycor, e = orc.heun_step(v0[0], v0[1], v1[0], v1[1], x, y, h)
    got_x = (xc + out[..., 0]).ravel()
    got_y = (yc + out[..., 1]).ravel()
    assert np.max(np.abs(got_x - xcor)) < tol * 10
    assert np.max(np.abs(got_y - ycor)) < tol * 10
    assert abs(err - e) < tol * 10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("L", [64, 128])
def test_integration_matches_oracle(orc, precision, L):
    m = _small_map(L=L, n=16 if L == 64 else 40)
    with _ctx(m, 1.0, precision) as c:
        c.spectrum()
        grid, acc, rej, t_end = c.integrate_once()
    spec = orc.forward(_oracle_density(orc, m), 1.0)
    r = orc.integrate(spec)
    assert r.status == 0
    tol = FP64_POS_TOL if precision == "fp64" else MIXED_POS_TOL
    if precision == "fp64":
        assert (acc, rej) == (r.accepted, r.rejected)
        assert t_end == pytest.approx(r.t_end, rel=1e-12)
    assert np.max(np.abs(grid[..., 0] - r.X)) < tol
    assert np.max(np.abs(grid[..., 1] - r.Y)) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_cartogram_matches_oracle(orc, precision):
    m = synth.make_workload("voronoi16_64")
    with _ctx(m, 1.0, precision) as c:
        st = c.integrate()
        xy = c.vertices()
        err = c.area_errors()
        nhist = c.history_length()
    r = orc.cartogram(m, blur=1.0)
    assert r.converged and st.converged
    assert st.iterations == r.iterations == nhist
    tol = FP64_POS_TOL if precision == "fp64" else MIXED_POS_TOL
    assert np.max(np.abs(xy - r.xy)) < tol
    assert np.max(np.abs(err - r.err)) < AREA_TOL
    assert st.max_area_error < 0.01
    if precision == "fp64":
        assert st.steps_accepted == r.steps_accepted and st.steps_rejected == r.steps_rejected


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_holes_and_islands_match_oracle(orc, precision):
    # a region with a hole (clockwise ring), a region filling the hole, and a region of two
    # islands listed apart in the ring order: densities, areas, and the whole cartogram
    m = synth.holes_map(64)
    with _ctx(m, 1.0, precision) as c:
        rho = c.density()
        err0 = c.area_errors()
        st = c.integrate()
        xy = c.vertices()
        err = c.area_errors()
        nhist = c.history_length()
    ref = _oracle_density(orc, m)
    assert np.max(np.abs(rho - ref)) < 1e-11 * np.max(np.abs(ref))
    A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, m.xy)
    assert np.allclose(A, [32 * 32 - 12 * 12, 12 * 12 + 12 * 14, 12 * 12, 48 * 12], rtol=1e-14)
    assert np.max(np.abs(err0 - (A / (m.values * A.sum() / m.values.sum()) - 1.0))) < 1e-13
    r = orc.cartogram(m, blur=1.0)
    assert r.converged and st.converged
    assert st.iterations == r.iterations == nhist
    tol = FP64_POS_TOL if precision == "fp64" else MIXED_POS_TOL
    assert np.max(np.abs(xy - r.xy)) < tol
    assert np.max(np.abs(err - r.err)) < AREA_TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("L", [64, 256])
def test_step_loop_modes_agree(precision, L):
    # persistent cooperative kernel, conditional CUDA graph and host-driven loop run the
    # same arithmetic: identical step counts and vertices
    m = _small_map(L=L, n=16 if L == 64 else 60)
    out = []
    for mode in (2, 1, 0):
        with _ctx(m, 1.0, precision, use_graph=mode) as c:
            s = c.integrate()
            out.append((s.iterations, s.steps_accepted, s.steps_rejected, c.vertices()))
    for o in out[1:]:
        assert o[:3] == out[0][:3]
        assert np.max(np.abs(o[3] - out[0][3])) < 1e-12


def test_project_reproduces_vertices_and_accepts_device_arrays():
    import torch
    m = _small_map()
    with _ctx(m, 1.0, "mixed") as c:
        c.integrate()
        xy = c.vertices()
        got = c.project(m.xy)
        assert np.max(np.abs(got - xy)) < 1e-12
        dev_in = torch.tensor(m.xy, device="cuda")
        dev_out = torch.empty_like(dev_in)
        P.cartogram_project(c.ctx, dev_in, dev_out)
        assert np.max(np.abs(dev_out.cpu().numpy() - xy)) < 1e-12
        assert c.project(np.zeros((0, 2))).shape == (0, 2)


def test_project_matches_oracle_composition(orc):
    m = _small_map()
    rng = np.random.default_rng(9)
    pts = np.stack([rng.uniform(0, m.Lx, 500), rng.uniform(0, m.Ly, 500)], axis=1)
    with _ctx(m, 1.0, "fp64") as c:
        c.integrate()
        got = c.project(pts)
        grids = [c.grid(k) for k in range(c.history_length())]
    r = orc.cartogram(m, blur=1.0)
    ref = pts.copy()
    for g in r.grids:
        ref = orc.map_points(g[0], g[1], ref)
    assert np.max(np.abs(got - ref)) < FP64_POS_TOL
    for g, go in zip(grids, r.grids):
        assert np.max(np.abs(g[..., 0] - go[0])) < FP64_POS_TOL
        assert np.max(np.abs(g[..., 1] - go[1])) < FP64_POS_TOL


def test_uniform_density_is_identity():
    # all regions at their target areas: no iteration, the map is unchanged
    m = synth.strip_map(32, 32, [0, 8, 16, 32], [8.0, 8.0, 16.0], spacing=1.0)
    with _ctx(m, 1.0, "fp64") as c:
        st = c.integrate()
        assert st.iterations == 0 and st.converged
        assert np.array_equal(c.vertices(), m.xy)


def test_strip_map_reaches_one_dimensional_solution():
    Lx, Ly = 64, 16
    V = [1.0, 3.0]
    m = synth.strip_map(Lx, Ly, [0, 32, 64], V, spacing=1.0)
    with _ctx(m, 0.0, "mixed") as c:
        st = c.integrate()
        xy = c.vertices()
    assert st.converged
    mid = np.abs(m.xy[:, 0] - 32.0) < 1e-12
    assert np.max(np.abs(xy[mid, 0] - Lx * V[0] / sum(V))) < 0.01 * Lx
    assert np.max(np.abs(xy[:, 1] - m.xy[:, 1])) < 1e-5


def test_invalid_inputs_are_rejected():
    m = _small_map()
    with P.Cartogram(64, 64, 1.0) as c:
        bad = m.values.copy()
        bad[3] = float("nan")
        for vals, off, reg, xy in (
            (bad, m.ring_offsets, m.ring_region, m.xy),
            (-m.values, m.ring_offsets, m.ring_region, m.xy),
            (m.values, m.ring_offsets, m.ring_region, m.xy + 60.0),
            (m.values, np.array([0, 2], dtype=np.int64), np.array([0], dtype=np.int32), m.xy[:2]),
            (m.values[:1], m.ring_offsets, m.ring_region, m.xy),
        ):
            with pytest.raises(P.CartogramError) as e:
                c.set_regions(vals, off, reg, xy)
            assert e.value.code == P.CG_EINVAL
        with pytest.raises(P.CartogramError) as e:
            c.integrate()
        assert e.value.code == P.CG_ESTATE
        # a clockwise-only region has negative area
        ring = synth.rectangle_ring(10, 10, 20, 20, 1.0)[::-1].copy()
        with pytest.raises(P.CartogramError) as e:
            c.set_regions(np.array([1.0]), np.array([0, len(ring)]), np.array([0], dtype=np.int32), ring)
        assert e.value.code == P.CG_EINVAL


def test_step_budget_exhaustion_reports_stepfail():
    m = _small_map()
    with _ctx(m, 1.0, "fp64", max_steps=3) as c:
        with pytest.raises(P.CartogramError) as e:
            c.integrate()
        assert e.value.code == P.CG_ESTEPFAIL
        # the map was left as it was
        assert np.array_equal(c.vertices(), m.xy)


def test_iteration_budget_reports_noconverge():
    m = _small_map()
    with _ctx(m, 1.0, "mixed", max_iter=2) as c:
        with pytest.raises(P.CartogramError) as e:
            c.integrate()
        assert e.value.code == P.CG_ENOCONVERGE
        assert c.history_length() == 2


@pytest.mark.parametrize("use_graph", [0, 1, 2])
def test_time_limit_reports_timeout(use_graph):
    # a 1 ns limit has passed by the first controller check: the integration in flight
    # ends with CG_ETIMEOUT and maps nothing; a generous limit changes nothing
    # (no autotuning: the first call then runs the device-side loop at once)
    m = _small_map()
    with _ctx(m, 1.0, "fp64", use_graph=use_graph, time_limit=1e-9, autotune=0) as c:
        with pytest.raises(P.CartogramError) as e:
            c.integrate()
        assert e.value.code == P.CG_ETIMEOUT
        assert np.array_equal(c.vertices(), m.xy) and c.history_length() == 0
        # entries other than cartogram_integrate do not use the limit
        loss, gv, gb = c.iteration_gradient(m.values, 1.0, 1e-3)
        assert np.isfinite(loss) and np.all(np.isfinite(gv))
    with _ctx(m, 1.0, "fp64", use_graph=use_graph) as c:
        st0 = c.integrate()
        xy0 = c.vertices()
    with _ctx(m, 1.0, "fp64", use_graph=use_graph, time_limit=100.0) as c:
        st1 = c.integrate()
        assert (st1.iterations, st1.steps_accepted, st1.steps_rejected) == \
            (st0.iterations, st0.steps_accepted, st0.steps_rejected)
        assert np.max(np.abs(c.vertices() - xy0)) < 1e-12


def test_grid_barrier_give_up_reports_timeout():
    """The persistent kernel's grid-barrier waits are bounded: with a one-poll limit the
    first barrier that is not already open makes its waiting blocks give up; every other
    block gives up at its next barrier, so the launch ends, the integration reports
    CG_ETIMEOUT and maps nothing. A generous limit reproduces the default run."""
    m = _small_map()
    with _ctx(m, 1.0, "fp64", use_graph=2, autotune=0) as ref:
        st0 = ref.integrate()
        xy0 = ref.vertices()
    with _ctx(m, 1.0, "fp64", use_graph=2, barrier_spins=1, autotune=0) as c:
        with pytest.raises(P.CartogramError) as e:
            c.integrate()
        assert e.value.code == P.CG_ETIMEOUT
        assert np.array_equal(c.vertices(), m.xy) and c.history_length() == 0
    # a context whose limit is generous reproduces the unlimited run
    with _ctx(m, 1.0, "fp64", use_graph=2, barrier_spins=1 << 30, autotune=0) as c:
        st1 = c.integrate()
        assert (st1.iterations, st1.steps_accepted, st1.steps_rejected) == \
            (st0.iterations, st0.steps_accepted, st0.steps_rejected)
        assert np.max(np.abs(c.vertices() - xy0)) < 1e-12


def test_time_limit_in_a_batch_and_in_the_linear_flow():
    m = _small_map()
    limited = P.Cartogram(m.Lx, m.Ly, 1.0, precision="mixed", time_limit=1e-9, autotune=0)
    free = P.Cartogram(m.Lx, m.Ly, 1.0, precision="mixed")
    lin = P.Cartogram(m.Lx, m.Ly, 4.0, precision="mixed", flow="linear", time_limit=1e-9)
    try:
        for c in (limited, free, lin):
            c.set_map(m)
        with P.Batch([limited, free]) as b:
            stats, status = b.integrate(check=False)
        assert status == [P.CG_ETIMEOUT, P.CG_OK]
        assert stats[1].converged and np.array_equal(limited.vertices(), m.xy)
        with pytest.raises(P.CartogramError) as e:
            lin.integrate()
        assert e.value.code == P.CG_ETIMEOUT
    finally:
        for c in (limited, free, lin):
            c.close()


@pytest.mark.parametrize("use_graph", [1, 2])
def test_a_map_with_the_same_rings_reuses_the_context(use_graph):
    # setting a map whose rings equal the current ones keeps the device buffers and the
    # captured graphs; the results must equal a fresh context's
    import dataclasses
    m = _small_map()
    rng = np.random.default_rng(3)
    m2 = dataclasses.replace(m, values=m.values * rng.lognormal(0.0, 0.5, m.n_regions))
    with _ctx(m, 1.0, "fp64", use_graph=use_graph) as c:
        st1 = c.integrate()
        xy1 = c.vertices()
        c.set_map(m2)
        assert c.history_length() == 0 and np.array_equal(c.vertices(), m2.xy)
        st2 = c.integrate()
        xy2 = c.vertices()
        c.set_map(m)
        st3 = c.integrate()
        assert (st3.iterations, st3.steps_accepted, st3.steps_rejected) == \
            (st1.iterations, st1.steps_accepted, st1.steps_rejected)
        assert np.max(np.abs(c.vertices() - xy1)) < 1e-10
        # other rings: a new map from scratch
        m3 = _small_map(L=64, n=12)
        c.set_map(m3)
        st4 = c.integrate()
        assert st4.converged
    with _ctx(m2, 1.0, "fp64", use_graph=use_graph) as c:
        st = c.integrate()
        assert (st.iterations, st.steps_accepted, st.steps_rejected) == \
            (st2.iterations, st2.steps_accepted, st2.steps_rejected)
        assert np.max(np.abs(c.vertices() - xy2)) < 1e-10


def test_set_values_restarts_from_the_original_map(orc):
    import dataclasses
    m = _small_map()
    rng = np.random.default_rng(4)
    v2 = m.values * rng.lognormal(0.0, 0.5, m.n_regions)
    with _ctx(m, 1.0, "fp64") as c:
        c.integrate()
        c.set_values(v2)
        assert c.history_length() == 0 and np.array_equal(c.vertices(), m.xy)
        A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, m.xy)
        assert np.max(np.abs(c.area_errors() - (A / (v2 * A.sum() / v2.sum()) - 1.0))) < 1e-13
        with pytest.raises(P.CartogramError) as e:
            c.set_values(-v2)
        assert e.value.code == P.CG_EINVAL
        st = c.integrate()
        xy = c.vertices()
    with _ctx(dataclasses.replace(m, values=v2), 1.0, "fp64") as c:
        st2 = c.integrate()
        assert (st.iterations, st.steps_accepted, st.steps_rejected) == \
            (st2.iterations, st2.steps_accepted, st2.steps_rejected)
        assert np.max(np.abs(xy - c.vertices())) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_square_cartogram_matches_oracle(orc, precision):
    # a 4 x 2 arrangement of rectangles on a 128 x 64 grid: every stage with Lx != Ly
    m = synth.blocks_map(128, 64)
    with _ctx(m, 1.0, precision) as c:
        st = c.integrate()
        xy = c.vertices()
        err = c.area_errors()
    r = orc.cartogram(m, blur=1.0)
    assert r.converged and st.converged and st.iterations == r.iterations
    tol = FP64_POS_TOL if precision == "fp64" else MIXED_POS_TOL
    assert np.max(np.abs(xy - r.xy)) < tol
    assert np.max(np.abs(err - r.err)) < AREA_TOL
    if precision == "fp64":
        assert st.steps_accepted == r.steps_accepted and st.steps_rejected == r.steps_rejected


def test_caller_stream_profile_and_autotune():
    # the context's work on a caller's stream gives the same result as on its own; the
    # kernel timings and the launch-shape tuner answer with sane values
    import torch
    m = _small_map(L=128, n=40)
    with _ctx(m, 1.0, "mixed") as c:
        st0 = c.integrate()
        xy0 = c.vertices()
    s = torch.cuda.Stream()
    with _ctx(m, 1.0, "mixed") as c:
        c.set_stream(s)
        st = c.integrate()
        assert (st.iterations, st.steps_accepted, st.steps_rejected) == \
            (st0.iterations, st0.steps_accepted, st0.steps_rejected)
        assert np.max(np.abs(c.vertices() - xy0)) < 1e-4  # atomic-order rounding of the FP32 path
        prof = c.profile(reps=3)
        assert set(prof) == set(P.PROFILE_CLASSES) and all(0.0 < v < 100.0 for v in prof.values())
        tuned = c.autotune(reps=2)
        assert tuned["rows_per_block"] >= 1 and tuned["cols_per_block"] >= 2 and tuned["heun_blocks_per_sm"] >= 1
        assert all(0.0 < v < 100.0 for v in tuned["ms"])
        st2 = c.integrate()  # converged already: no iteration
        assert st2.iterations == 0


@pytest.mark.parametrize("use_graph", [0, 1])
def test_iteration_records(orc, use_graph):
    """Per-iteration records of the history (largest area error after the iteration, its
    end time, step counts, device time, blur width) in both outer-loop modes, against
    the oracle run for one and two iterations."""
    m = _small_map()
    with _ctx(m, 1.0, "fp64", use_graph=use_graph) as c:
        st = c.integrate()
        recs = c.iteration_history()
    assert len(recs) == st.iterations
    assert recs[-1]["max_area_error"] == pytest.approx(st.max_area_error, rel=1e-12)
    assert sum(r["steps_accepted"] for r in recs) == st.steps_accepted
    assert sum(r["steps_rejected"] for r in recs) == st.steps_rejected
    for k, r in enumerate(recs):
        assert r["blur"] == pytest.approx(1.0 * 0.5 ** k, rel=1e-15)
        assert r["step_loop_ms"] > 0 and r["t_end"] > 0
    for k in (1, 2):
        ref = orc.cartogram(m, 1.0, keep_grids=False, max_iter=k)
        assert recs[k - 1]["max_area_error"] == pytest.approx(ref.max_area_error, abs=1e-9)
        assert sum(r["steps_accepted"] for r in recs[:k]) == ref.steps_accepted
        assert sum(r["steps_rejected"] for r in recs[:k]) == ref.steps_rejected
    with _ctx(m, 1.0, "fp64", use_graph=use_graph) as c:
        with pytest.raises(P.CartogramError) as e:
            c.iteration_record(0)  # no history yet
        assert e.value.code == P.CG_EINVAL
