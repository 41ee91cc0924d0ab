"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself:
brute-force double sums, closed forms of the diffusion flow, invariants and
hand-computed geometry. Each test names the passage of the paper it pins.
"""
import math

import numpy as np
import pytest

from paper_1802_07625_gb300 import synth

PI = math.pi


# --------------------------------------------------------------------------
# brute force on tiny grids (pure Python, math.cos evaluated directly)
# --------------------------------------------------------------------------

def brute_forward(rho, blur):
    """Main text Eq. rhotilde_mn with the integral as a midpoint sum, 4-fold loop."""
    Ly, Lx = rho.shape
    out = np.zeros((Ly, Lx))
    for n in range(Ly):
        for m in range(Lx):
            s = 0.0
            for j in range(Ly):
                for i in range(Lx):
                    s += rho[j, i] * math.cos(PI * m * (i + 0.5) / Lx) * math.cos(PI * n * (j + 0.5) / Ly)
            w = 4.0 / ((1 + (m == 0)) * (1 + (n == 0)))
            k2 = m * m / Lx ** 2 + n * n / Ly ** 2
            out[n, m] = w * s * math.exp(-PI * PI * blur * blur * k2 / 2)
    return out


def brute_fields(spec, t):
    """SI Eq. rhoxyt with f_mn = exp(-pi^2 (m^2/Lx^2 + n^2/Ly^2) t) and its x/y derivatives."""
    Ly, Lx = spec.shape
    rho = np.zeros((Ly, Lx))
    gx = np.zeros((Ly, Lx))
    gy = np.zeros((Ly, Lx))
    for j in range(Ly):
        y = j + 0.5
        for i in range(Lx):
            x = i + 0.5
            r = a = b = 0.0
            for n in range(Ly):
                for m in range(Lx):
                    c = spec[n, m] * math.exp(-PI * PI * (m * m / Lx ** 2 + n * n / Ly ** 2) * t)
                    r += c * math.cos(PI * m * x / Lx) * math.cos(PI * n * y / Ly)
                    a += c * (-PI * m / Lx) * math.sin(PI * m * x / Lx) * math.cos(PI * n * y / Ly)
                    b += c * math.cos(PI * m * x / Lx) * (-PI * n / Ly) * math.sin(PI * n * y / Ly)
            rho[j, i] = r / (Lx * Ly)
            gx[j, i] = a / (Lx * Ly)
            gy[j, i] = b / (Lx * Ly)
    return rho, gx, gy


@pytest.mark.parametrize("shape", [(8, 8), (6, 8), (8, 6)])
@pytest.mark.parametrize("blur", [0.0, 1.3])
def test_forward_matches_brute_force(orc, shape, blur):
    rng = np.random.default_rng(11)
    rho = rng.uniform(0.2, 3.0, size=shape)
    got = orc.forward(rho, blur)
    ref = brute_forward(rho, blur)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(8, 8), (6, 8)])
@pytest.mark.parametrize("t", [0.0, 0.37])
def test_fields_match_brute_force(orc, shape, t):
    rng = np.random.default_rng(12)
    spec = rng.standard_normal(shape)
    rho, gx, gy = orc.fields(spec, t)
    r0, a0, b0 = brute_fields(spec, t)
    for got, ref in ((rho, r0), (gx, a0), (gy, b0)):
        assert np.max(np.abs(got - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(16, 12), (64, 64), (10, 32)])
def test_round_trip_is_identity(orc, shape):
    # the inverse series of SI Eq. rhoxyt undoes the coefficients of Eq. rhotilde_mn
    # exactly on the cell-centre grid (discrete orthogonality of the cosines)
    rng = np.random.default_rng(13)
    rho = rng.uniform(0.1, 5.0, size=shape)
    back, _, _ = orc.fields(orc.forward(rho, 0.0), 0.0)
    assert np.max(np.abs(back - rho)) < 1e-13 * np.max(rho)


def test_single_mode_has_one_coefficient(orc):
    Ly, Lx = 12, 16
    x = np.arange(Lx) + 0.5
    y = np.arange(Ly) + 0.5
    rho = np.cos(2 * PI * x[None, :] / Lx) * np.cos(PI * y[:, None] / Ly)
    spec = orc.forward(rho, 0.0)
    expect = np.zeros((Ly, Lx))
    expect[1, 2] = Lx * Ly  # 4 * (Lx/2) * (Ly/2)
    assert np.max(np.abs(spec - expect)) < 1e-11


def test_mean_coefficient_is_total_mass(orc):
    # SI: rho~_00 = rho_bar Lx Ly
    rng = np.random.default_rng(14)
    rho = rng.uniform(0.1, 5.0, size=(20, 24))
    spec = orc.forward(rho, 2.0)
    assert abs(spec[0, 0] - rho.sum()) < 1e-11 * rho.sum()


def test_blur_is_gaussian_of_width_sigma(orc):
    # a Gaussian blur of standard deviation sigma multiplies the coefficient of
    # wavenumber k = pi m / L by exp(-k^2 sigma^2 / 2)
    Ly, Lx = 8, 32
    x = np.arange(Lx) + 0.5
    rho = 1.0 + 0.3 * np.cos(3 * PI * x / Lx)[None, :] * np.ones((Ly, 1))
    s0 = orc.forward(rho, 0.0)
    s1 = orc.forward(rho, 1.7)
    k = 3 * PI / Lx
    assert abs(s1[0, 3] / s0[0, 3] - math.exp(-k * k * 1.7 ** 2 / 2)) < 1e-13
    assert abs(s1[0, 0] - s0[0, 0]) < 1e-12 * s0[0, 0]


# --------------------------------------------------------------------------
# closed form of the diffusion flow for one cosine mode
# --------------------------------------------------------------------------

@pytest.mark.parametrize("t", [0.0, 3.0, 40.0])
def test_single_mode_decay_and_velocity(orc, t):
    # rho0 = 1 + a cos(pi x / Lx): SI Eq. fmn_diff (D = 1 time) gives
    # rho = 1 + a e^{-pi^2 t/Lx^2} cos(pi x/Lx), v_x = -d_x rho / rho, v_y = 0
    Ly, Lx, a = 8, 32, 0.4
    x = np.arange(Lx) + 0.5
    rho0 = (1 + a * np.cos(PI * x / Lx))[None, :] * np.ones((Ly, 1))
    spec = orc.forward(rho0, 0.0)
    rho, gx, gy = orc.fields(spec, t)
    decay = math.exp(-PI * PI * t / Lx ** 2)
    rho_ref = 1 + a * decay * np.cos(PI * x / Lx)
    gx_ref = -a * decay * (PI / Lx) * np.sin(PI * x / Lx)
    assert np.max(np.abs(rho - rho_ref[None, :])) < 1e-13
    assert np.max(np.abs(gx - gx_ref[None, :])) < 1e-13
    assert np.max(np.abs(gy)) < 1e-13
    vx, vy, vmax = orc.velocity(rho, gx, gy)
    vx_ref = -gx_ref / rho_ref
    assert np.max(np.abs(vx - vx_ref[None, :])) < 1e-13
    assert np.max(np.abs(vy)) < 1e-13
    assert abs(vmax - np.max(np.abs(vx_ref))) < 1e-13


def test_two_dimensional_mode_decay_rate(orc):
    # mode (m, n) = (2, 3) decays as exp(-pi^2 (4/Lx^2 + 9/Ly^2) t)
    Ly, Lx, t = 12, 16, 2.5
    spec = np.zeros((Ly, Lx))
    spec[3, 2] = 5.0
    rho, gx, gy = orc.fields(spec, t)
    x = np.arange(Lx) + 0.5
    y = np.arange(Ly) + 0.5
    f = 5.0 * math.exp(-PI * PI * (4 / Lx ** 2 + 9 / Ly ** 2) * t) / (Lx * Ly)
    cx, cy = np.cos(2 * PI * x / Lx), np.cos(3 * PI * y / Ly)
    sx, sy = np.sin(2 * PI * x / Lx), np.sin(3 * PI * y / Ly)
    assert np.max(np.abs(rho - f * cy[:, None] * cx[None, :])) < 1e-15
    assert np.max(np.abs(gx - f * cy[:, None] * (-2 * PI / Lx) * sx[None, :])) < 1e-15
    assert np.max(np.abs(gy - f * (-3 * PI / Ly) * sy[:, None] * cx[None, :])) < 1e-15


# --------------------------------------------------------------------------
# interpolation and the no-flux walls
# --------------------------------------------------------------------------

def _linear_field(Lx, Ly, A, b):
    x = np.arange(Lx) + 0.5
    y = np.arange(Ly) + 0.5
    X, Y = np.meshgrid(x, y)
    vx = A[0][0] * X + A[0][1] * Y + b[0]
    vy = A[1][0] * X + A[1][1] * Y + b[1]
    return vx, vy


def test_interp_reproduces_linear_fields_inside(orc):
    Lx, Ly = 10, 7
    A = [[0.3, -0.2], [0.15, 0.4]]
    b = [0.7, -0.5]
    vx, vy = _linear_field(Lx, Ly, A, b)
    rng = np.random.default_rng(3)
    for _ in range(50):
        x = rng.uniform(0.5, Lx - 0.5)
        y = rng.uniform(0.5, Ly - 0.5)
        ux, uy = orc.interp(vx, vy, x, y)
        assert abs(ux - (A[0][0] * x + A[0][1] * y + b[0])) < 1e-13
        assert abs(uy - (A[1][0] * x + A[1][1] * y + b[1])) < 1e-13


def test_interp_at_grid_points_and_walls(orc):
    Lx, Ly = 9, 6
    rng = np.random.default_rng(4)
    vx = rng.standard_normal((Ly, Lx))
    vy = rng.standard_normal((Ly, Lx))
    for j in range(Ly):
        for i in range(Lx):
            ux, uy = orc.interp(vx, vy, i + 0.5, j + 0.5)
            assert ux == pytest.approx(vx[j, i], abs=1e-15)
            assert uy == pytest.approx(vy[j, i], abs=1e-15)
    for y in np.linspace(0, Ly, 13):
        # no flux through the walls x = 0 and x = Lx (main text: no flow through the
        # edges of the box)
        assert orc.interp(vx, vy, 0.0, y)[0] == 0.0
        assert orc.interp(vx, vy, float(Lx), y)[0] == 0.0
    for x in np.linspace(0, Lx, 13):
        assert orc.interp(vx, vy, x, 0.0)[1] == 0.0
        assert orc.interp(vx, vy, x, float(Ly))[1] == 0.0
    # tangential component on a wall equals the nearest grid point's
    j = 2
    assert orc.interp(vx, vy, 0.0, j + 0.5)[1] == pytest.approx(vy[j, 0], abs=1e-15)
    assert orc.interp(vx, vy, float(Lx), j + 0.5)[1] == pytest.approx(vy[j, Lx - 1], abs=1e-15)
    # halfway between the wall and the first grid point the normal component is halved
    assert orc.interp(vx, vy, 0.25, j + 0.5)[0] == pytest.approx(0.5 * vx[j, 0], abs=1e-15)


# --------------------------------------------------------------------------
# predictor-corrector step
# --------------------------------------------------------------------------

def test_heun_step_closed_form_for_linear_fields(orc):
    # For v0(r) = A r + b and v1(r) = c (A r + b), Heun's step is
    #   r* = r + h (A r + b),  r' = r + h/2 ((A r + b) + c (A r* + b))
    Lx, Ly = 40, 30
    A = np.array([[0.02, -0.01], [0.015, -0.03]])
    b = np.array([0.1, -0.05])
    c = 1.7
    v0x, v0y = _linear_field(Lx, Ly, A, b)
    v1x, v1y = c * v0x, c * v0y
    rng = np.random.default_rng(5)
    pts = np.stack([rng.uniform(10, 30, 40), rng.uniform(8, 22, 40)], axis=1)
    h = 0.8
    xp, yp, xc, yc, err = orc.heun_step(v0x, v0y, v1x, v1y, pts[:, 0].copy(), pts[:, 1].copy(), h)
    f0 = pts @ A.T + b
    rstar = pts + h * f0
    f1 = c * (rstar @ A.T + b)
    rcorr = pts + 0.5 * h * (f0 + f1)
    assert np.max(np.abs(np.stack([xp, yp], 1) - rstar)) < 1e-13
    assert np.max(np.abs(np.stack([xc, yc], 1) - rcorr)) < 1e-13
    assert err == pytest.approx(np.max(np.linalg.norm(rcorr - rstar, axis=1)), rel=1e-12)


def test_heun_step_stays_in_box(orc):
    Lx, Ly = 8, 8
    vx = np.full((Ly, Lx), 5.0)
    vy = np.full((Ly, Lx), -5.0)
    x = np.array([7.6])
    y = np.array([0.3])
    _, _, xc, yc, _ = orc.heun_step(vx, vy, vx, vy, x, y, 1.0)
    assert 0.0 <= xc[0] <= Lx and 0.0 <= yc[0] <= Ly


# --------------------------------------------------------------------------
# the integration
# --------------------------------------------------------------------------

def test_uniform_density_gives_identity(orc):
    Ly, Lx = 16, 24
    spec = orc.forward(np.full((Ly, Lx), 2.5), 1.0)
    r = orc.integrate(spec)
    x = np.arange(Lx) + 0.5
    y = np.arange(Ly) + 0.5
    assert r.accepted == 0 and r.status == 0
    assert np.array_equal(r.X, np.broadcast_to(x[None, :], (Ly, Lx)))
    assert np.array_equal(r.Y, np.broadcast_to(y[:, None], (Ly, Lx)))


def test_x_only_density_gives_one_dimensional_equalising_map(orc):
    # SI Eq. det in one dimension has the unique monotone solution
    #   T_x(x) = (1/rho_bar) int_0^x rho0,  T_y = y.
    # For rho0 = 1 + a cos(pi x / L): T_x = x + (a L / pi) sin(pi x / L).
    Ly, Lx, a = 8, 64, 0.5
    x = np.arange(Lx) + 0.5
    rho0 = (1 + a * np.cos(PI * x / Lx))[None, :] * np.ones((Ly, 1))
    spec = orc.forward(rho0, 0.0)
    exact = x + a * Lx / PI * np.sin(PI * x / Lx)
    errs = []
    for atol in (4e-2, 1e-2, 2.5e-3):
        r = orc.integrate(spec, atol=atol, rho_tol=1e-7)
        assert r.status == 0
        assert np.max(np.abs(r.Y - (np.arange(Ly) + 0.5)[:, None])) == 0.0
        errs.append(np.max(np.abs(r.X - exact[None, :])))
    # second-order scheme: the error falls with the step tolerance and is small
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.03


def _one_mode_spectrum(orc, Ly=8, Lx=64, a=0.5):
    x = np.arange(Lx) + 0.5
    rho0 = (1 + a * np.cos(PI * x / Lx))[None, :] * np.ones((Ly, 1))
    return orc.forward(rho0, 0.0)


def test_heun_is_second_order_in_time(orc):
    # The predictor-corrector (Eq. rt_diff integrated by Heun's method) on a fixed schedule
    # of n equal steps to the same end time, against 1024 steps with the same field and
    # interpolation: halving the step quarters the error (global error O(h^2)). A first-
    # order slip (e.g. the corrector dropping v(t + h)) would give ratios near 2.
    spec = _one_mode_spectrum(orc)
    T = 200.0

    def run(n):
        return orc.integrate_replay(spec, [T / n] * n)[0]

    ref = run(1024)
    e = [np.max(np.abs(run(n) - ref)) for n in (8, 16, 32)]
    for coarse, fine in zip(e, e[1:]):
        assert 3.7 < coarse / fine < 4.3, e


def test_adaptive_error_scales_with_the_step_tolerance(orc):
    # The step error r_corr - r_pred = (h/2)(u1 - u0) is O(h^2), so with acceptance at
    # e <= atol the steps scale as atol^(1/2) and the time-integration error (against a
    # fine fixed schedule to the same end time, same field and interpolation) as atol:
    # a quarter of atol gives about a quarter of the error.
    spec = _one_mode_spectrum(orc)
    errs = []
    for atol in (4e-2, 1e-2, 2.5e-3):
        r = orc.integrate(spec, atol=atol, rho_tol=1e-7)
        assert r.status == 0
        ref = orc.integrate_replay(spec, [r.t_end / 4096] * 4096)[0]
        errs.append(np.max(np.abs(r.X - ref)))
        # the recorded schedule obeys the controller: a rejected step is retried at half
        # its size, an accepted one grows by at most 1.2 (less where the speed cap holds),
        # and the accepted steps add up to the end time
        h, acc = r.sched_h, r.sched_acc.astype(bool)
        assert np.sum(h[acc]) == pytest.approx(r.t_end, rel=1e-12)
        for k in range(len(h) - 1):
            if acc[k]:
                assert h[k + 1] <= 1.2 * h[k] * (1 + 1e-15)
            else:
                assert h[k + 1] == pytest.approx(0.5 * h[k], rel=1e-15)
    for coarse, fine in zip(errs, errs[1:]):
        assert 2.5 < coarse / fine < 5.0, errs


def test_adaptive_heun_follows_a_brute_force_rk4_trajectory(orc):
    # Brute force on an 8x8 grid: every grid point's trajectory dr/dt = v(r, t) (main text
    # Eq. rt_diff) integrated by classical RK4 with 400 equal steps to the adaptive
    # integration's own end time, through the same fields and interpolation. The RK4
    # solution is converged (200 against 400 steps agree to ~1e-6), so the difference is
    # the adaptive predictor-corrector's time-integration error: within about atol, and
    # falling with it. A slip in the step, the controller or the time bookkeeping (a
    # stage at the wrong time, an accepted step whose time is not advanced) shows here.
    L = 8
    c = np.arange(L) + 0.5
    X0, Y0 = np.meshgrid(c, c)
    rho = (1 + 0.4 * np.cos(PI * X0 / L) * np.cos(PI * Y0 / L) + 0.25 * np.cos(2 * PI * Y0 / L)
           + 0.2 * np.cos(3 * PI * X0 / L))
    spec = orc.forward(rho, 0.0)

    def vel(t, px, py):
        vx, vy, _ = orc.velocity(*orc.fields(spec, t))
        u = np.array([orc.interp(vx, vy, a, b) for a, b in zip(px, py)])
        return u[:, 0], u[:, 1]

    def rk4(T, n):
        px, py, h = X0.ravel().copy(), Y0.ravel().copy(), T / n
        for k in range(n):
            t = k * h
            k1 = vel(t, px, py)
            k2 = vel(t + h / 2, px + h / 2 * k1[0], py + h / 2 * k1[1])
            k3 = vel(t + h / 2, px + h / 2 * k2[0], py + h / 2 * k2[1])
            k4 = vel(t + h, px + h * k3[0], py + h * k3[1])
            px = px + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
            py = py + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        return px.reshape(L, L), py.reshape(L, L)

    errs = []
    for atol in (1e-2, 1e-3, 1e-4):
        r = orc.integrate(spec, atol=atol, rho_tol=1e-4)
        assert r.status == 0
        xr, yr = rk4(r.t_end, 400)
        assert np.max(np.abs(xr - X0)) > 0.3  # the points do move
        e = max(np.max(np.abs(r.X - xr)), np.max(np.abs(r.Y - yr)))
        assert e < 1.5 * atol, (atol, e)
        errs.append(e)
    assert errs[0] > 3 * errs[1] > 9 * errs[2]


def test_mirror_symmetry(orc):
    rng = np.random.default_rng(6)
    Ly, Lx = 12, 12
    rho0 = rng.uniform(0.5, 2.0, (Ly, Lx))
    r1 = orc.integrate(orc.forward(rho0, 1.0))
    r2 = orc.integrate(orc.forward(rho0[:, ::-1].copy(), 1.0))
    assert r1.accepted == r2.accepted
    assert np.max(np.abs(r2.X[:, ::-1] - (Lx - r1.X))) < 1e-9
    assert np.max(np.abs(r2.Y[:, ::-1] - r1.Y)) < 1e-9


def test_transpose_symmetry(orc):
    rng = np.random.default_rng(7)
    L = 12
    rho0 = rng.uniform(0.5, 2.0, (L, L))
    r1 = orc.integrate(orc.forward(rho0, 1.0))
    r2 = orc.integrate(orc.forward(rho0.T.copy(), 1.0))
    assert np.max(np.abs(r2.X.T - r1.Y)) < 1e-9
    assert np.max(np.abs(r2.Y.T - r1.X)) < 1e-9


def test_projected_grid_has_positive_jacobian(orc):
    m = synth.make_workload("voronoi16_64")
    A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, m.xy)
    rho = orc.rasterize(m.Lx, m.Ly, m.values, A, m.ring_offsets, m.ring_region, m.xy)
    r = orc.integrate(orc.forward(rho, 1.0))
    X, Y = r.X, r.Y
    # signed area of every quad of projected cell centres (no fold-overs)
    ax = X[:-1, 1:] - X[:-1, :-1]
    ay = Y[:-1, 1:] - Y[:-1, :-1]
    bx = X[1:, :-1] - X[:-1, :-1]
    by = Y[1:, :-1] - Y[:-1, :-1]
    assert np.min(ax * by - ay * bx) > 0.0


# --------------------------------------------------------------------------
# geometry: areas, rasterisation, point mapping
# --------------------------------------------------------------------------

def test_region_areas_and_orientation(orc):
    sq = [[1, 1], [3, 1], [3, 3], [1, 3]]                 # CCW, area 4
    hole = [[1.5, 1.5], [1.5, 2.0], [2.0, 2.0], [2.0, 1.5]]  # CW, area -0.25
    tri = [[5, 5], [8, 5], [5, 9]]                         # CCW, area 6
    xy = np.array(sq + hole + tri, dtype=float)
    offs = np.array([0, 4, 8, 11])
    reg = np.array([0, 0, 1], dtype=np.int32)
    A = orc.region_areas(2, offs, reg, xy)
    assert A[0] == pytest.approx(3.75, abs=1e-14)
    assert A[1] == pytest.approx(6.0, abs=1e-14)
    err, mx = orc.area_errors(np.array([1.0, 3.0]), A)
    # targets: V_i * sum(A) / sum(V) = 9.75/4 * [1, 3]
    assert err[0] == pytest.approx(3.75 / (9.75 / 4) - 1, abs=1e-14)
    assert err[1] == pytest.approx(6.0 / (9.75 * 3 / 4) - 1, abs=1e-14)
    assert mx == pytest.approx(max(abs(err[0]), abs(err[1])), abs=0)


def _overlap(a0, a1, b0, b1):
    return max(0.0, min(a1, b1) - max(a0, b0))


def test_rasterize_rectangles_exact_coverage(orc):
    Lx, Ly = 8, 6
    r1 = (1.25, 0.5, 3.5, 4.75)
    r2 = (4.0, 1.2, 7.3, 5.0)
    ring1 = synth.rectangle_ring(*r1, spacing=0.7)
    ring2 = synth.rectangle_ring(*r2, spacing=0.45)
    xy = np.concatenate([ring1, ring2])
    offs = np.array([0, len(ring1), len(ring1) + len(ring2)])
    reg = np.array([0, 1], dtype=np.int32)
    vals = np.array([2.0, 7.0])
    A = orc.region_areas(2, offs, reg, xy)
    a1 = (r1[2] - r1[0]) * (r1[3] - r1[1])
    a2 = (r2[2] - r2[0]) * (r2[3] - r2[1])
    assert A == pytest.approx([a1, a2], abs=1e-13)
    rho = orc.rasterize(Lx, Ly, vals, A, offs, reg, xy)
    d_out = vals.sum() / (a1 + a2)
    for j in range(Ly):
        for i in range(Lx):
            c1 = _overlap(i, i + 1, r1[0], r1[2]) * _overlap(j, j + 1, r1[1], r1[3])
            c2 = _overlap(i, i + 1, r2[0], r2[2]) * _overlap(j, j + 1, r2[1], r2[3])
            ref = d_out + (vals[0] / a1 - d_out) * c1 + (vals[1] / a2 - d_out) * c2
            assert rho[j, i] == pytest.approx(ref, abs=1e-13)
    # the box's mean density is the map's mean density
    assert rho.mean() == pytest.approx(d_out, rel=1e-13)


def test_rasterize_triangle_and_hole(orc):
    # right triangle (0,0),(4,0),(0,4): cells below the diagonal are full, cells the
    # diagonal cuts through are half covered; a clockwise square ring removes area
    Lx, Ly = 6, 6
    tri = np.array([[0, 0], [4, 0], [0, 4]], dtype=float)
    hole = np.array([[0.5, 0.5], [0.5, 1.5], [1.5, 1.5], [1.5, 0.5]], dtype=float)
    other = synth.rectangle_ring(4.0, 4.0, 6.0, 6.0, 1.0)
    xy = np.concatenate([tri, hole, other])
    offs = np.array([0, 3, 7, 7 + len(other)])
    reg = np.array([0, 0, 1], dtype=np.int32)
    vals = np.array([3.0, 1.0])
    A = orc.region_areas(2, offs, reg, xy)
    assert A[0] == pytest.approx(8.0 - 1.0)
    rho = orc.rasterize(Lx, Ly, vals, A, offs, reg, xy)
    d_out = vals.sum() / A.sum()
    w0 = vals[0] / A[0] - d_out
    w1 = vals[1] / A[1] - d_out
    for j in range(Ly):
        for i in range(Lx):
            cov = 1.0 if i + j + 2 <= 4 else (0.5 if i + j == 3 else 0.0)
            cov -= _overlap(i, i + 1, 0.5, 1.5) * _overlap(j, j + 1, 0.5, 1.5)
            cov1 = 1.0 if (i >= 4 and j >= 4) else 0.0
            assert rho[j, i] == pytest.approx(d_out + w0 * cov + w1 * cov1, abs=1e-13)


def test_rasterize_voronoi_total_mass(orc):
    m = synth.make_workload("voronoi16_64")
    A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, m.xy)
    rho = orc.rasterize(m.Lx, m.Ly, m.values, A, m.ring_offsets, m.ring_region, m.xy)
    d_out = m.values.sum() / A.sum()
    # sum over cells of rho = d_out * box area (the margin carries the mean density)
    assert rho.sum() == pytest.approx(d_out * m.Lx * m.Ly, rel=1e-12)
    # the inset margin is exactly d_out
    assert np.all(rho[:8, :] == d_out) and np.all(rho[:, :8] == d_out)
    assert np.all(rho > 0)


def test_map_points_identity_and_affine(orc):
    Lx, Ly = 12, 9
    x = np.arange(Lx) + 0.5
    y = np.arange(Ly) + 0.5
    X, Y = np.meshgrid(x, y)
    rng = np.random.default_rng(8)
    pts = np.stack([rng.uniform(0, Lx, 200), rng.uniform(0, Ly, 200)], axis=1)
    out = orc.map_points(X, Y, pts)
    assert np.max(np.abs(out - pts)) < 1e-13
    # an affine projected grid maps every point affinely (bilinear reproduces affine maps,
    # inside and in the extended half-cell band along the walls)
    M = np.array([[1.1, 0.2], [-0.1, 0.9]])
    c = np.array([0.3, -0.4])
    Xa = M[0, 0] * X + M[0, 1] * Y + c[0]
    Ya = M[1, 0] * X + M[1, 1] * Y + c[1]
    out = orc.map_points(Xa, Ya, pts)
    assert np.max(np.abs(out - (pts @ M.T + c))) < 1e-12


# --------------------------------------------------------------------------
# the whole method
# --------------------------------------------------------------------------

def test_strip_map_converges_to_one_dimensional_solution(orc):
    # two vertical strips that tile the box: the density is x-only, so the converged
    # cartogram moves the dividing line to x = Lx V0 / (V0 + V1) (SI Eq. det in 1-D)
    Lx, Ly = 32, 16
    V = [1.0, 3.0]
    m = synth.strip_map(Lx, Ly, [0, 16, 32], V, spacing=1.0)
    r = orc.cartogram(m, blur=0.0)
    assert r.converged and r.status == 0
    assert r.max_area_error < 0.01
    xy = r.xy
    mid = np.abs(m.xy[:, 0] - 16.0) < 1e-12
    target = Lx * V[0] / sum(V)
    assert np.max(np.abs(xy[mid, 0] - target)) < 0.01 * Lx
    # nothing moves vertically in an x-only flow
    assert np.max(np.abs(xy[:, 1] - m.xy[:, 1])) < 1e-12


def test_voronoi_map_converges(orc):
    m = synth.make_workload("voronoi16_64")
    r = orc.cartogram(m, blur=1.0)
    assert r.converged and r.max_area_error < 0.01
    # every region's area is within 1% of its target; the sum of target areas is the
    # sum of current areas by construction
    A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, r.xy)
    err, mx = orc.area_errors(m.values, A)
    assert mx == pytest.approx(r.max_area_error)


# --------------------------------------------------------------------------
# the linear-equalisation flow (SI Eq. fmn_fast, f_mn = 1 - t)
# --------------------------------------------------------------------------

def test_linear_flux_single_mode_closed_form(orc):
    # rho0 = 1 + a cos(pi x / Lx): J_x = (a Lx / pi) sin(pi x / Lx), J_y = 0, so that
    # -d_x J_x = -a cos(pi x/Lx) = rho_bar - rho0 (continuity with rho(t) = (1-t) rho0 + t)
    Ly, Lx, a = 8, 32, 0.4
    x = np.arange(Lx) + 0.5
    rho0 = (1 + a * np.cos(PI * x / Lx))[None, :] * np.ones((Ly, 1))
    jx, jy = orc.flux_linear(orc.forward(rho0, 0.0))
    assert np.max(np.abs(jx - (a * Lx / PI * np.sin(PI * x / Lx))[None, :])) < 1e-12
    assert np.max(np.abs(jy)) < 1e-13


def test_linear_flux_two_dimensional_mode(orc):
    # one coefficient c at (m, n) = (2, 3): SI Eqs. Jxmn, Jymn with f' = -1 and Eqs. Jx, Jy
    Ly, Lx, c = 12, 16, 5.0
    spec = np.zeros((Ly, Lx))
    spec[3, 2] = c
    jx, jy = orc.flux_linear(spec)
    x = np.arange(Lx) + 0.5
    y = np.arange(Ly) + 0.5
    den = PI * (4 * Ly ** 2 + 9 * Lx ** 2)
    jxm = 2 * Lx * Ly ** 2 * c / den / (Lx * Ly)
    jym = 3 * Lx ** 2 * Ly * c / den / (Lx * Ly)
    assert np.max(np.abs(jx - jxm * np.cos(3 * PI * y / Ly)[:, None] * np.sin(2 * PI * x / Lx)[None, :])) < 1e-15
    assert np.max(np.abs(jy - jym * np.sin(3 * PI * y / Ly)[:, None] * np.cos(2 * PI * x / Lx)[None, :])) < 1e-15


def test_linear_flux_satisfies_continuity(orc):
    # a smooth 2-D density: the central-difference divergence of J matches rho0 - rho_bar
    # to the second-order truncation error of the differences
    L = 64
    x = np.arange(L) + 0.5
    X, Y = np.meshgrid(x, x)
    rho0 = 1 + 0.3 * np.cos(PI * X / L) * np.cos(2 * PI * Y / L) + 0.2 * np.cos(3 * PI * Y / L)
    jx, jy = orc.flux_linear(orc.forward(rho0, 0.0))
    div = (jx[1:-1, 2:] - jx[1:-1, :-2]) / 2 + (jy[2:, 1:-1] - jy[:-2, 1:-1]) / 2
    err = np.max(np.abs(div - (rho0[1:-1, 1:-1] - rho0.mean())))
    assert err < 0.01 and err > 0.0
    # curl-free: d_y J_x = d_x J_y (SI Eq. novortex)
    curl = (jx[2:, 1:-1] - jx[:-2, 1:-1]) / 2 - (jy[1:-1, 2:] - jy[1:-1, :-2]) / 2
    assert np.max(np.abs(curl)) < 1e-3


def test_linear_flow_reaches_one_dimensional_map_at_t_one(orc):
    Ly, Lx, a = 8, 64, 0.5
    x = np.arange(Lx) + 0.5
    rho0 = (1 + a * np.cos(PI * x / Lx))[None, :] * np.ones((Ly, 1))
    spec = orc.forward(rho0, 0.0)
    exact = x + a * Lx / PI * np.sin(PI * x / Lx)
    errs = []
    for atol in (4e-2, 1e-2, 2.5e-3):
        r = orc.integrate_linear(spec, atol=atol)
        assert r.status == 0 and r.t_end == 1.0
        # the n >= 1 coefficients of an x-only density are rounding noise
        assert np.max(np.abs(r.Y - (np.arange(Ly) + 0.5)[:, None])) < 1e-12
        errs.append(np.max(np.abs(r.X - exact[None, :])))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.03


def test_linear_flow_strip_map_converges(orc):
    Lx, Ly = 32, 16
    V = [1.0, 3.0]
    m = synth.strip_map(Lx, Ly, [0, 16, 32], V, spacing=1.0)
    r = orc.cartogram(m, blur=0.0, flow=1)
    assert r.converged and r.max_area_error < 0.01
    mid = np.abs(m.xy[:, 0] - 16.0) < 1e-12
    assert np.max(np.abs(r.xy[mid, 0] - Lx * V[0] / sum(V))) < 0.01 * Lx


# ---------------------------------------------------------------------------------
# diagnostics of the composed projection: Tissot distortion (SI section 3) and the
# inverse map (the main text's inverse graticule)
# ---------------------------------------------------------------------------------

def _affine_grid(L, A, b):
    x = np.arange(L) + 0.5
    X, Y = np.meshgrid(x, x)
    return np.stack([A[0, 0] * X + A[0, 1] * Y + b[0], A[1, 0] * X + A[1, 1] * Y + b[1]])


def _tissot(A):
    s = np.linalg.svd(A, compute_uv=False)
    return np.log(s[0] / s[1]), 2 * np.arcsin((s[0] - s[1]) / (s[0] + s[1]))


def test_distortion_of_affine_and_composed_grids(orc):
    # a bilinear grid of an affine map is that map everywhere (its quads extended too):
    # the Jacobian is A, constant, so mean = max = the closed-form Tissot measures
    L = 16
    A1 = np.array([[2.0, 0.3], [0.1, 0.8]])
    A2 = np.array([[0.7, -0.2], [0.4, 1.3]])
    g1 = _affine_grid(L, A1, [0.2, -0.1])
    g2 = _affine_grid(L, A2, [-1.0, 0.5])
    e, et = _tissot(A1)
    assert np.allclose(orc.distortion(g1[None]), [e, e, et, et], rtol=0, atol=1e-12)
    # composition: T2(T1(r)) has the constant Jacobian A2 A1
    e, et = _tissot(A2 @ A1)
    assert np.allclose(orc.distortion(np.stack([g1, g2])), [e, e, et, et], rtol=0, atol=1e-12)
    # identity and a pure rotation are conformal
    assert np.allclose(orc.distortion(_affine_grid(L, np.eye(2), [0, 0])[None]), 0.0, atol=1e-12)
    c, s = np.cos(0.4), np.sin(0.4)
    assert np.allclose(orc.distortion(_affine_grid(L, np.array([[c, -s], [s, c]]), [3, 1])[None]), 0.0, atol=1e-12)


def test_distortion_chain_rule_matches_finite_differences(orc):
    # on the grids of a real cartogram: e at each quad centre from the chain-rule Jacobian
    # agrees with the Jacobian of the composed point map by central differences
    m = synth.make_workload("voronoi16_64", L=32, n=10)
    r = orc.cartogram(m, blur=1.0)
    g = r.grids
    L = m.Lx
    xc = np.arange(1, L) * 1.0
    P0 = np.stack(np.meshgrid(xc, xc), axis=-1).reshape(-1, 2)
    h = 1e-6

    def T(p):
        for k in range(g.shape[0]):
            p = orc.map_points(g[k, 0], g[k, 1], p)
        return p

    Jx = (T(P0 + [h, 0]) - T(P0 - [h, 0])) / (2 * h)
    Jy = (T(P0 + [0, h]) - T(P0 - [0, h])) / (2 * h)
    J = np.stack([Jx, Jy], axis=-1)  # [n][2 (T component)][2 (d/dx, d/dy)]
    s = np.linalg.svd(J, compute_uv=False)
    e = np.log(s[:, 0] / s[:, 1])
    et = 2 * np.arcsin((s[:, 0] - s[:, 1]) / (s[:, 0] + s[:, 1]))
    d = orc.distortion(g)
    assert abs(d[0] - e.mean()) < 1e-6 and abs(d[1] - e.max()) < 1e-6
    assert abs(d[2] - et.mean()) < 1e-6 and abs(d[3] - et.max()) < 1e-6
    assert d[1] > 0.1  # the map is not conformal


def test_inverse_points_of_affine_grids(orc):
    # maps that keep the box's points inside the box, as the cartogram's grids do (the
    # inverse looks for preimages inside the box)
    L = 16
    A1 = np.array([[0.9, 0.05], [0.05, 0.85]])
    A2 = np.array([[0.95, -0.05], [0.05, 0.9]])
    b1, b2 = np.array([0.5, 0.8]), np.array([0.6, 0.4])
    g = np.stack([_affine_grid(L, A1, b1), _affine_grid(L, A2, b2)])
    rng = np.random.default_rng(11)
    p = rng.uniform(1.0, L - 1.0, (50, 2))
    q = (A2 @ (A1 @ p.T + b1[:, None]) + b2[:, None]).T
    assert np.max(np.abs(orc.inverse_points(g, q) - p)) < 1e-10


def test_inverse_points_undo_the_cartograms_point_map(orc):
    # round trip through orc_map_points on the grids of a real cartogram, including
    # points in the half-cell band along the walls
    m = synth.make_workload("voronoi16_64", L=32, n=10)
    g = orc.cartogram(m, blur=1.0).grids
    rng = np.random.default_rng(12)
    p = np.concatenate([rng.uniform(0.0, m.Lx, (300, 2)), [[0.1, 0.2], [31.9, 0.3], [0.25, 31.8], [31.95, 31.9]]])
    q = p.copy()
    for k in range(g.shape[0]):
        q = orc.map_points(g[k, 0], g[k, 1], q)
    back = orc.inverse_points(g, q)
    assert np.max(np.abs(back - p)) < 1e-9
    # a point outside the image of the box has no preimage
    assert np.all(np.isnan(orc.inverse_points(g, np.array([[-5.0, 3.0]]))))


# ---------------------------------------------------------------------------------
# FP64 reverse-mode reference of one outer iteration's loss (oracle/adjoint.py)
# ---------------------------------------------------------------------------------

def _adjoint_case(orc, L=32, n=8):
    import torch

    from oracle import adjoint as adj
    m = synth.make_workload("voronoi16_64", L=L, n=n)
    A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, m.xy)
    it = adj.Iteration(m, orc.coverage(m), A)
    blur = 1.0
    with torch.no_grad():
        spec_t = it.spectrum(torch.tensor(m.values), torch.tensor(blur, dtype=torch.float64))
    rho_p = np.tensordot(m.values / A * (A.sum() / m.values.sum()) - 1.0, orc.coverage(m), 1)
    r = orc.integrate(orc.forward(1.0 + rho_p, blur))
    return adj, m, A, it, blur, spec_t, r


def test_adjoint_forward_replays_the_oracle_integration(orc):
    import torch
    adj, m, A, it, blur, spec_t, r = _adjoint_case(orc)
    spec_c = orc.forward(1.0 + np.tensordot(m.values / A * (A.sum() / m.values.sum()) - 1.0, orc.coverage(m), 1), blur)
    s = spec_t.numpy()
    assert np.max(np.abs(s.ravel()[1:] - spec_c.ravel()[1:])) < 1e-11 * np.max(np.abs(spec_c))
    steps = adj.accepted_steps(r.sched_h, r.sched_acc)
    assert len(steps) == r.accepted
    with torch.no_grad():
        X, Y = it.integrate(spec_t, steps)
    assert np.max(np.abs(X.numpy() - r.X)) < 1e-10 and np.max(np.abs(Y.numpy() - r.Y)) < 1e-10
    # the loss as the oracle's own functions give it
    lam = 1e-3
    xy1 = orc.map_points(r.X, r.Y, m.xy)
    A1 = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, xy1)
    target = m.values * A1.sum() / m.values.sum()
    ref = np.sum((np.log(A1) - np.log(target)) ** 2) + lam * np.sum((xy1 - m.xy) ** 2)
    with torch.no_grad():
        L, _ = it.loss(torch.tensor(m.values), torch.tensor(blur, dtype=torch.float64), steps, lam)
    assert abs(float(L) - ref) < 1e-10 * abs(ref)


def test_adjoint_gradient_matches_central_differences(orc):
    import torch
    adj, m, A, it, blur, spec_t, r = _adjoint_case(orc)
    steps = adj.accepted_steps(r.sched_h, r.sched_acc)
    lam = 1e-3
    L, gv, gs = adj.gradient(it, m.values, blur, steps, lam)

    def loss(values, b):
        with torch.no_grad():
            return float(it.loss(torch.tensor(values), torch.tensor(b, dtype=torch.float64), steps, lam)[0])

    for i in (0, 3, m.n_regions - 1):
        h = 1e-6 * m.values[i]
        vp, vm = m.values.copy(), m.values.copy()
        vp[i] += h
        vm[i] -= h
        fd = (loss(vp, blur) - loss(vm, blur)) / (2 * h)
        assert abs(fd - gv[i]) <= 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(gv))), (i, fd, gv[i])
    h = 1e-6
    fd = (loss(m.values, blur + h) - loss(m.values, blur - h)) / (2 * h)
    assert abs(fd - gs) <= 1e-6 * abs(fd)
    assert np.max(np.abs(gv)) > 0 and gs != 0


def test_multi_iteration_oracle_loss_reduces_to_the_reference(orc):
    # one iteration of the C-oracle loss with the replayed schedule equals the autograd
    # reference's loss (itself pinned to the oracle's integration above)
    import torch
    adj, m, A, it, blur, spec_t, r = _adjoint_case(orc)
    steps = adj.accepted_steps(r.sched_h, r.sched_acc)
    sch = adj.adaptive_schedules(orc, m, m.values, blur, 0.5, 2)
    assert sch[0] == steps and len(sch[1]) > 0
    with torch.no_grad():
        L_t, _ = it.loss(torch.tensor(m.values), torch.tensor(blur, dtype=torch.float64), steps, 1e-3)
    L_c = adj.cartogram_loss(orc, m, m.values, blur, 0.5, [steps], 1e-3)
    assert abs(L_c - float(L_t)) < 1e-10 * abs(L_c)
    # a second iteration moves the areas further towards their targets
    L_2 = adj.cartogram_loss(orc, m, m.values, blur, 0.5, sch, 0.0)
    L_1 = adj.cartogram_loss(orc, m, m.values, blur, 0.5, sch[:1], 0.0)
    assert L_2 < L_1


# ---- polygon-level measures (SI section 4) ------------------------------------------


def _rot(xy, beta, centre=(5.0, 4.0)):
    c = np.asarray(centre)
    R = np.array([[math.cos(beta), -math.sin(beta)], [math.sin(beta), math.cos(beta)]])
    return (xy - c) @ R.T + c


def test_centroids_of_a_rectangle_and_a_square_with_a_hole():
    from oracle import polygon as pg
    outer = synth.rectangle_ring(0, 0, 4, 4, 1.0)
    hole = synth.rectangle_ring(0, 0, 2, 2, 1.0)[::-1]
    rect = synth.rectangle_ring(5, 1, 9, 3, 0.5)
    xy = np.concatenate([outer, hole, rect])
    off = np.cumsum([0, len(outer), len(hole), len(rect)])
    c = pg.region_centroids(2, off, np.array([0, 0, 1]), xy)
    # [0,4]^2 minus [0,2]^2: (16 (2,2) - 4 (1,1)) / 12 = (7/3, 7/3)
    assert np.allclose(c, [[7 / 3, 7 / 3], [7.0, 2.0]], atol=1e-14)


def test_relative_position_error_of_similarity_maps():
    from oracle import polygon as pg
    m = synth.make_workload("voronoi16_64", L=32, n=8)
    c = pg.region_centroids(m.n_regions, m.ring_offsets, m.ring_region, m.xy)
    assert pg.relative_position_error(c, c) == 0.0
    # translations and uniform scalings keep every direction: theta = 0
    assert pg.relative_position_error(c, 0.5 * c + 3.0) < 1e-15
    # a rotation by beta turns every connecting line by beta: theta = beta / pi
    for beta in (0.1, 1.0, 2.5):
        d = pg.region_centroids(m.n_regions, m.ring_offsets, m.ring_region, _rot(m.xy, beta))
        assert abs(pg.relative_position_error(c, d) - beta / math.pi) < 1e-12


def test_aspect_ratio_of_rectangles_and_a_hexagon():
    from oracle import polygon as pg
    rect = synth.rectangle_ring(1, 1, 4, 2, 0.25)  # 3 x 1
    for beta in (0.0, 0.3, 1.2):
        hull = pg.convex_hull(_rot(rect, beta))
        area, alpha = pg.min_area_rectangle(hull)
        assert abs(area - 3.0) < 1e-12 and abs(alpha - 3.0) < 1e-12
    hexagon = np.array([[math.cos(k * math.pi / 3), math.sin(k * math.pi / 3)] for k in range(6)])
    # every orientation along a side gives the 2 x sqrt(3) rectangle
    area, alpha = pg.min_area_rectangle(pg.convex_hull(_rot(hexagon, 0.4, (0, 0))))
    assert abs(area - 2 * math.sqrt(3)) < 1e-12 and abs(alpha - 2 / math.sqrt(3)) < 1e-12


def test_aspect_ratio_matches_a_brute_force_scan_over_orientations():
    from oracle import polygon as pg
    # a non-convex star: its hull's edges bridge the concavities
    k = np.arange(14)
    rad = np.where(k % 2 == 0, 3.0, 1.2) * (1.0 + 0.15 * np.sin(k))
    star = np.stack([10 + rad * np.cos(2 * math.pi * k / 14) * 1.7, 10 + rad * np.sin(2 * math.pi * k / 14)], 1)
    area, alpha = pg.min_area_rectangle(pg.convex_hull(star))
    phi = np.linspace(0.0, math.pi / 2, 20001)[:-1]
    u = np.stack([np.cos(phi), np.sin(phi)], 1)
    a = star @ u.T
    b = star @ np.stack([-np.sin(phi), np.cos(phi)], 1).T
    w, t = a.max(0) - a.min(0), b.max(0) - b.min(0)
    j = np.argmin(w * t)
    assert area <= (w * t)[j] + 1e-12 and (w * t)[j] - area < 1e-3 * area
    assert abs(max(w[j], t[j]) / min(w[j], t[j]) - alpha) < 1e-3 * alpha


def test_aspect_ratio_ties_go_to_the_smaller_ratio():
    from oracle import polygon as pg
    # region 3 of the 64^2 Voronoi map is cut by two sides of the inset square: two hull
    # edges give the same minimum area with different aspect ratios
    m = synth.make_workload("voronoi16_64")
    pts = m.xy[m.ring_offsets[3]:m.ring_offsets[4]]
    hull = pg.convex_hull(pts)
    cands = []
    for e in range(len(hull)):
        u = hull[(e + 1) % len(hull)] - hull[e]
        u = u / np.hypot(*u)
        w = np.ptp(hull @ u)
        t = np.ptp(hull @ np.array([-u[1], u[0]]))
        cands.append((w * t, max(w, t) / min(w, t)))
    amin = min(a for a, _ in cands)
    tied = sorted(r for a, r in cands if a <= amin * (1 + 1e-9))
    assert len(tied) >= 2 and tied[-1] - tied[0] > 0.1
    area, alpha = pg.min_area_rectangle(hull)
    assert area == amin and alpha == tied[0]
