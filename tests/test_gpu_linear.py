"""The linear-equalisation flow (SI Eq. fmn_fast: rho(t) = (1-t) rho0 + t rho_bar, a
constant flux from SI Eqs. Jxmn and Jymn, integration to t = 1) on the GPU against the
oracle's linear integration and its whole cartogram with flow = 1, through the C-ABI.
Tolerances as for the diffusion flow: 1e-9 grid units (FP64 path), 1e-3 (mixed path),
identical accept/reject counts on the FP64 path."""
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


def _maps():
    # square Voronoi maps spanning several tiles, and a strip map with Lx != Ly (the
    # flux weights m/Lx and n/Ly differ)
    yield "voronoi64", synth.make_workload("voronoi16_64", L=64, n=16)
    yield "voronoi128", synth.make_workload("voronoi16_64", L=128, n=40)
    yield "strips128x32", synth.strip_map(128, 32, [0, 32, 64, 128], [1.0, 3.0, 0.5], spacing=0.6)


MAPS = dict(_maps())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(MAPS))
def test_linear_integration_matches_oracle(orc, precision, name):
    m = MAPS[name]
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision=precision, flow="linear") as c:
        c.set_map(m)
        c.spectrum()
        grid, acc, rej, t_end = c.integrate_once()
    r = orc.integrate_linear(orc.forward(_oracle_density(orc, m), 1.0))
    assert r.status == 0 and r.t_end == 1.0
    assert t_end == 1.0
    if precision == "fp64":
        assert (acc, rej) == (r.accepted, r.rejected)
    tol = FP64_POS_TOL if precision == "fp64" else MIXED_POS_TOL
    assert np.max(np.abs(grid[..., 0] - r.X)) < tol
    assert np.max(np.abs(grid[..., 1] - r.Y)) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linear_cartogram_matches_oracle(orc, precision):
    m = synth.make_workload("voronoi16_64")
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision=precision, flow="linear") as c:
        c.set_map(m)
        st = c.integrate()
        xy = c.vertices()
        err = c.area_errors()
    r = orc.cartogram(m, blur=1.0, flow=1)
    assert r.converged and st.converged
    assert st.iterations == r.iterations
    assert st.t_end == 1.0
    tol = FP64_POS_TOL if precision == "fp64" else MIXED_POS_TOL
    assert np.max(np.abs(xy - r.xy)) < tol
    assert np.max(np.abs(err - r.err)) < AREA_TOL
    if precision == "fp64":
        assert st.steps_accepted == r.steps_accepted and st.steps_rejected == r.steps_rejected


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linear_loop_modes_agree(precision):
    # conditional CUDA graph, host-driven loop, and the persistent option (which runs the
    # graph for this flow): the same kernels and the same results
    m = synth.make_workload("voronoi16_64", L=128, n=40)
    out = []
    for mode in (1, 0, 2):
        with P.Cartogram(m.Lx, m.Ly, 1.0, precision=precision, flow="linear", use_graph=mode) as c:
            c.set_map(m)
            s = c.integrate()
            out.append((s.iterations, s.steps_accepted, s.steps_rejected, c.vertices()))
    for o in out[1:]:
        assert o[:3] == out[0][:3]
        assert np.max(np.abs(o[3] - out[0][3])) < 1e-12


def test_linear_strip_map_reaches_one_dimensional_solution():
    # two strips of values 1 and 3: the shared boundary moves to x = Lx/4, heights stay
    Lx, Ly = 64, 16
    V = [1.0, 3.0]
    m = synth.strip_map(Lx, Ly, [0, 32, 64], V, spacing=1.0)
    with P.Cartogram(Lx, Ly, 0.0, precision="mixed", flow="linear") as c:
        c.set_map(m)
        st = c.integrate()
        xy = c.vertices()
    assert st.converged
    mid = np.abs(m.xy[:, 0] - 32.0) < 1e-12
    assert np.max(np.abs(xy[mid, 0] - Lx * V[0] / sum(V))) < 0.01 * Lx
    assert np.max(np.abs(xy[:, 1] - m.xy[:, 1])) < 1e-5


def test_linear_step_budget_reports_stepfail():
    m = synth.make_workload("voronoi16_64")
    for mode in (1, 0):
        with P.Cartogram(m.Lx, m.Ly, 1.0, flow="linear", max_steps=5, use_graph=mode) as c:
            c.set_map(m)
            with pytest.raises(P.CartogramError) as e:
                c.integrate()
            assert e.value.code == P.CG_ESTEPFAIL
