"""Parity at the workloads' full sizes (512^2 and 1024^2), through the C-ABI, in the launch
configuration the benchmark uses. The oracle evaluates whole fields by direct sums
(O(L^3), seconds on the host cores) and single steps; a whole converged 1024^2 cartogram
is checked through properties that hold at any size."""
import numpy as np
import pytest

import paper_1802_07625_gb300 as P
from paper_1802_07625_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def big():
    return synth.make_workload("powerlaw3000_1024")


def _oracle_density(orc, m):
    A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, m.xy)
    rho = orc.rasterize(m.Lx, m.Ly, m.values, A, m.ring_offsets, m.ring_region, m.xy)
    return rho / (m.values.sum() / A.sum())


def test_density_spectrum_field_and_step_at_1024(orc, big):
    m = big
    blur = synth.WORKLOADS["powerlaw3000_1024"]["blur"]
    with P.Cartogram(m.Lx, m.Ly, blur, precision="mixed") as c:
        c.set_map(m)
        rho_gpu = c.density()
        spec_gpu = c.spectrum()
        t, h = 3.0, 0.8
        rho_t, v_t = c.velocity(t)
        rng = np.random.default_rng(3)
        disp = rng.uniform(-2.0, 2.0, (m.Ly, m.Lx, 2))
        out, err = c.heun_step(t, h, disp)
    rho0 = _oracle_density(orc, m)
    # the oracle's plain shoelace of clipped polygons at coordinates ~1e3, weighted by
    # densities up to ~1e5 rho_bar (Pareto values on sub-cell regions), rounds at ~1e-10
    # of the maximum; the GPU accumulates pieces relative to the cell edges
    assert np.max(np.abs(rho_gpu - rho0)) < 1e-9 * np.max(rho0)
    spec = orc.forward(rho0, blur)
    assert np.max(np.abs(spec_gpu - spec)) < 1e-11 * np.max(np.abs(spec))
    r0, gx, gy = orc.fields(spec, t)
    vx, vy, vmax = orc.velocity(r0, gx, gy)
    # FP32 transforms: absolute errors ~ eps32 log2(N) times the fields' global scale
    # (max|rho'| for rho, max|grad rho| for the gradient); v = -grad rho / rho divides by
    # the local density
    eps = 2.0 ** -24 * np.log2(m.Lx) * 8
    R = np.max(np.abs(r0 - 1.0))
    G = np.max(np.hypot(gx, gy))
    assert np.max(np.abs(rho_t - r0)) < eps * R
    bound = eps * (G + R * np.hypot(vx, vy)) / r0
    assert np.all(np.abs(v_t[..., 0] - vx) <= bound)
    assert np.all(np.abs(v_t[..., 1] - vy) <= bound)
    # one predictor-corrector step of all 1024^2 points from the same displacements
    v1 = orc.velocity(*orc.fields(spec, t + h))
    xc = np.arange(m.Lx)[None, :] + 0.5
    yc = np.arange(m.Ly)[:, None] + 0.5
    x = np.clip(xc + disp[..., 0], 0, m.Lx)
    y = np.clip(yc + disp[..., 1], 0, m.Ly)
    _, _, xcor, ycor, e = orc.heun_step(vx, vy, v1[0], v1[1], x.ravel(), y.ravel(), h)
    gx_ = (xc + out[..., 0]).ravel()
    gy_ = (yc + out[..., 1]).ravel()
    assert np.max(np.abs(gx_ - xcor)) < 1e-3
    assert np.max(np.abs(gy_ - ycor)) < 1e-3
    assert abs(err - e) < 1e-3


def _quad_areas(g):
    ax = g[:-1, 1:, 0] - g[:-1, :-1, 0]
    ay = g[:-1, 1:, 1] - g[:-1, :-1, 1]
    bx = g[1:, :-1, 0] - g[:-1, :-1, 0]
    by = g[1:, :-1, 1] - g[:-1, :-1, 1]
    return ax * by - ay * bx


def test_converged_1024_cartogram_properties(big):
    m = big
    blur = synth.WORKLOADS["powerlaw3000_1024"]["blur"]
    with P.Cartogram(m.Lx, m.Ly, blur, precision="mixed", max_iter=100) as c:
        c.set_map(m)
        st = c.integrate()
        xy = c.vertices()
        err = c.area_errors()
        grids = [c.grid(k) for k in range(c.history_length())]
        folds = [c.fold_count(k) for k in range(c.history_length())]
        proj = c.project(m.xy)
    assert st.converged and st.max_area_error < 0.01
    assert np.max(np.abs(err)) < 0.01
    for g, (nf, amin) in zip(grids, folds):
        # every projected grid stays in the box; the fold detector agrees with the grid
        assert g.min() >= 0.0 and g[..., 0].max() <= m.Lx and g[..., 1].max() <= m.Ly
        A = _quad_areas(g)
        assert nf == int(np.sum(A <= 0.0))
        assert amin == pytest.approx(float(A.min()), abs=1e-6)
    # The map has regions far below one cell (0.2 cells^2 at ~1e5 times the mean
    # density), which the grid does not resolve: the first integration folds a handful of
    # quads next to them (the FP64 path folds the same ones, see below); later ones do not.
    assert folds[0][0] < 1e-3 * (m.Lx - 1) * (m.Ly - 1)
    assert all(nf == 0 for nf, _ in folds[1:])
    # shared boundaries stay shared: the composed map is a function of the point
    assert np.max(np.abs(proj - xy)) < 1e-9
    A = np.array([0.5 * np.sum(xy[a:b, 0] * np.roll(xy[a:b, 1], -1) - np.roll(xy[a:b, 0], -1) * xy[a:b, 1])
                  for a, b in zip(m.ring_offsets[:-1], m.ring_offsets[1:])])
    target = m.values * A.sum() / m.values.sum()
    assert np.max(np.abs(A / target - 1.0)) < 0.01


def test_first_integration_folds_agree_between_precisions(big):
    m = big
    blur = synth.WORKLOADS["powerlaw3000_1024"]["blur"]
    out = {}
    for prec in ("fp64", "mixed"):
        with P.Cartogram(m.Lx, m.Ly, blur, precision=prec, max_iter=1) as c:
            c.set_map(m)
            with pytest.raises(P.CartogramError):
                c.integrate()  # one iteration does not converge
            out[prec] = (c.fold_count(0), c.grid(0))
    (n64, a64), g64 = out["fp64"]
    (n32, a32), g32 = out["mixed"]
    assert np.max(np.abs(g64 - g32)) < 1e-3
    assert n64 == n32
    assert a32 == pytest.approx(a64, abs=1e-2)


def test_first_integration_at_256_matches_oracle(orc):
    # the clustered recipe on a 256^2 grid: one whole integration, element by element
    m = synth.make_workload("clustered300_512", L=256, n=120)
    with P.Cartogram(m.Lx, m.Ly, 2.0, precision="mixed") as c:
        c.set_map(m)
        c.spectrum()
        grid, acc, rej, t_end = c.integrate_once()
    spec = orc.forward(_oracle_density(orc, m), 2.0)
    r = orc.integrate(spec)
    assert r.status == 0
    assert np.max(np.abs(grid[..., 0] - r.X)) < 1e-3
    assert np.max(np.abs(grid[..., 1] - r.Y)) < 1e-3


@pytest.fixture(scope="module")
def clustered():
    return synth.make_workload("clustered300_512")


def test_density_spectrum_field_and_step_at_512(orc, clustered):
    # the 512^2 clustered workload (lognormal(1.5) values, blur 2) in both precisions
    m = clustered
    blur = synth.WORKLOADS["clustered300_512"]["blur"]
    rho0 = _oracle_density(orc, m)
    spec = orc.forward(rho0, blur)
    t, h = 1.5, 0.6
    r0, gx, gy = orc.fields(spec, t)
    vx, vy, _ = orc.velocity(r0, gx, gy)
    v1 = orc.velocity(*orc.fields(spec, t + h))
    rng = np.random.default_rng(4)
    disp = rng.uniform(-1.5, 1.5, (m.Ly, m.Lx, 2))
    xc = np.arange(m.Lx)[None, :] + 0.5
    yc = np.arange(m.Ly)[:, None] + 0.5
    x = np.clip(xc + disp[..., 0], 0, m.Lx)
    y = np.clip(yc + disp[..., 1], 0, m.Ly)
    _, _, xcor, ycor, e = orc.heun_step(vx, vy, v1[0], v1[1], x.ravel(), y.ravel(), h)
    # field error bounds relative to the fields' global scale: FP32 transforms ~ eps32
    # log2(N) per value; the FP64 transforms and the oracle's direct sums both ~1e-14
    for prec, eps, ptol in (("fp64", 1e-12, 1e-9), ("mixed", 2.0 ** -24 * np.log2(m.Lx) * 8, 1e-3),
                            ("mixed_ff", 2.0 ** -24 * np.log2(m.Lx) * 8, 1e-3)):
        with P.Cartogram(m.Lx, m.Ly, blur, precision=prec) as c:
            c.set_map(m)
            rho_gpu = c.density()
            spec_gpu = c.spectrum()
            rho_t, v_t = c.velocity(t)
            out, err = c.heun_step(t, h, disp)
        assert np.max(np.abs(rho_gpu - rho0)) < 1e-9 * np.max(rho0)
        assert np.max(np.abs(spec_gpu - spec)) < 1e-11 * np.max(np.abs(spec))
        # the velocity divides by the local density
        R = np.max(np.abs(r0 - 1.0))
        G = np.max(np.hypot(gx, gy))
        assert np.max(np.abs(rho_t - r0)) < eps * R
        bound = eps * (G + R * np.hypot(vx, vy)) / r0
        assert np.all(np.abs(v_t[..., 0] - vx) <= bound)
        assert np.all(np.abs(v_t[..., 1] - vy) <= bound)
        assert np.max(np.abs((xc + out[..., 0]).ravel() - xcor)) < ptol
        assert np.max(np.abs((yc + out[..., 1]).ravel() - ycor)) < ptol
        assert abs(err - e) < ptol


def test_converged_512_cartogram_properties(clustered):
    m = clustered
    blur = synth.WORKLOADS["clustered300_512"]["blur"]
    with P.Cartogram(m.Lx, m.Ly, blur, precision="mixed") as c:
        c.set_map(m)
        st = c.integrate()
        xy = c.vertices()
        folds = [c.fold_count(k)[0] for k in range(c.history_length())]
        proj = c.project(m.xy)
    assert st.converged and st.max_area_error < 0.01
    # one region has a target of 2.3 cells^2 (about 1.5 cells wide): once the grid no
    # longer resolves it, it shrinks a few percent per iteration
    assert 100 < st.iterations < 500
    assert folds[0] < 1e-3 * (m.Lx - 1) * (m.Ly - 1)
    assert all(nf == 0 for nf in folds[1:])
    assert np.max(np.abs(proj - xy)) < 1e-9


def test_fp64_and_mixed_agree_on_first_integrations_at_512(clustered):
    # The FP64 path at 512^2 (its autotuner candidates are limited by the kernels'
    # register use) against the mixed path over two integrations with the same step
    # schedule. This map has regions at 0.0018 of the mean density next to peaks at 80:
    # FP32 transform round-off (~1e-6 of the global field scale) is ~20 % of the density
    # there, so points inside those regions drift until the diffusing mass arrives. The
    # drift stays below 1e-3 grid units for 99.9 % of the points and below 3e-3 for all;
    # FP32 displacements alone (FP64 fields) account for 1.4e-4 and the FP32 spectrum
    # alone for 6e-5.
    # With pass 2 in float-float arithmetic (precision "mixed_ff") every point is within 1e-3.
    m = clustered
    blur = synth.WORKLOADS["clustered300_512"]["blur"]
    out = {}
    for prec in ("fp64", "mixed", "mixed_ff"):
        with P.Cartogram(m.Lx, m.Ly, blur, precision=prec, max_iter=2) as c:
            c.set_map(m)
            with pytest.raises(P.CartogramError) as e:
                c.integrate()
            assert e.value.code == P.CG_ENOCONVERGE
            out[prec] = (c.grid(0), c.grid(1), c.area_errors())
    for k in range(2):
        d = np.abs(out["fp64"][k] - out["mixed"][k])
        assert np.mean(d > 1e-3) < 1e-3
        assert np.max(d) < 3e-3
        dff = np.abs(out["fp64"][k] - out["mixed_ff"][k])
        print("first integrations at 512^2, iteration %d: mixed %.3g, mixed_ff %.3g" % (k, d.max(), dff.max()))
        assert np.max(dff) < 1e-3
    assert np.max(np.abs(out["fp64"][2] - out["mixed"][2])) < 1e-4
    assert np.max(np.abs(out["fp64"][2] - out["mixed_ff"][2])) < 1e-4
