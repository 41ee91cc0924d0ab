"""Reverse-mode gradient of one outer iteration on the GPU (FP64 path), through the C-ABI:
against the FP64 reverse-mode reference of oracle/adjoint.py (same step schedule: the FP64
path and the oracle take the same accept/reject decisions) and against central finite
differences of the GPU's own loss with the schedule held fixed (replay). The loss is
sum_i (ln A'_i - ln A^_i)^2 + lam sum_v |X'_v - X_v|^2 of the mapped map."""
import numpy as np
import pytest

import paper_1802_07625_gb300 as P
from paper_1802_07625_gb300 import synth

pytestmark = pytest.mark.gpu
LAM = 1e-3


def _rel(a, b, scale):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / scale


@pytest.mark.parametrize("L,n", [(32, 8), (64, 16)])
def test_gradient_matches_fp64_reverse_mode_oracle(orc, L, n):
    import torch  # noqa: F401  (the reference uses torch's CPU autograd)

    from oracle import adjoint as adj
    m = synth.make_workload("voronoi16_64", L=L, n=n)
    blur = 1.0
    with P.Cartogram(L, L, blur, precision="fp64") as c:
        c.set_map(m)
        loss, gv, gb = c.iteration_gradient(m.values, blur, LAM)
        loss_replay = c.iteration_gradient(m.values, blur, LAM, replay=True, grad=False)
    A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, m.xy)
    it = adj.Iteration(m, orc.coverage(m), A)
    rho_p = np.tensordot(m.values / A * (A.sum() / m.values.sum()) - 1.0, orc.coverage(m), 1)
    r = orc.integrate(orc.forward(1.0 + rho_p, blur))
    steps = adj.accepted_steps(r.sched_h, r.sched_acc)
    L_ref, gv_ref, gb_ref = adj.gradient(it, m.values, blur, steps, LAM)
    assert abs(loss - L_ref) < 1e-9 * abs(L_ref)
    assert abs(loss_replay - loss) < 1e-12 * abs(loss)
    assert _rel(gv, gv_ref, np.max(np.abs(gv_ref))) < 1e-7
    assert abs(gb - gb_ref) < 1e-7 * abs(gb_ref)


def _fd_check(c, values, blur, g_v, g_b, regions, h_rel, tol):
    for i in regions:
        h = h_rel * values[i]
        vp, vm = values.copy(), values.copy()
        vp[i] += h
        vm[i] -= h
        fd = (c.iteration_gradient(vp, blur, LAM, replay=True, grad=False)
              - c.iteration_gradient(vm, blur, LAM, replay=True, grad=False)) / (2 * h)
        assert abs(fd - g_v[i]) <= tol * max(abs(fd), 1e-3 * np.max(np.abs(g_v))), (i, fd, g_v[i])
    h = h_rel * blur
    fd = (c.iteration_gradient(values, blur + h, LAM, replay=True, grad=False)
          - c.iteration_gradient(values, blur - h, LAM, replay=True, grad=False)) / (2 * h)
    assert abs(fd - g_b) <= tol * abs(fd), (fd, g_b)


def test_gradient_matches_central_differences_at_64():
    m = synth.make_workload("voronoi16_64")
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="fp64") as c:
        c.set_map(m)
        loss, gv, gb = c.iteration_gradient(m.values, 1.0, LAM, checkpoint=5)
        _fd_check(c, m.values, 1.0, gv, gb, [0, 7, 15], 1e-5, 1e-6)
        # the checkpoint spacing changes nothing but the recomputation
        _, gv2, gb2 = c.iteration_gradient(m.values, 1.0, LAM, replay=True, checkpoint=1)
        assert np.max(np.abs(gv2 - gv)) <= 1e-12 * np.max(np.abs(gv)) and abs(gb2 - gb) <= 1e-12 * abs(gb)
        # the map itself is unchanged
        assert np.array_equal(c.vertices(), m.xy) and c.history_length() == 0


@pytest.mark.slow
def test_gradient_at_512_against_central_differences():
    # the differentiation workload: the 512^2 clustered map with lognormal(1.5) values,
    # blur 2, checkpoints every 8 steps; central differences with h = 1e-4 (relative)
    m = synth.make_workload("clustered300_512")
    blur = synth.WORKLOADS["clustered300_512"]["blur"]
    rng = np.random.default_rng(31)
    with P.Cartogram(m.Lx, m.Ly, blur, precision="fp64") as c:
        c.set_map(m)
        loss, gv, gb = c.iteration_gradient(m.values, blur, LAM, checkpoint=8)
        assert np.all(np.isfinite(gv)) and np.isfinite(gb) and loss > 0
        regions = rng.choice(m.n_regions, 6, replace=False).tolist() + [int(np.argmax(np.abs(gv)))]
        _fd_check(c, m.values, blur, gv, gb, regions, 1e-4, 1e-4)


def test_gradient_rejects_what_it_cannot_do():
    m = synth.make_workload("voronoi16_64")
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="mixed") as c:
        c.set_map(m)
        with pytest.raises(P.CartogramError) as e:
            c.iteration_gradient(m.values, 1.0)
        assert e.value.code == P.CG_EINVAL
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="fp64") as c:
        c.set_map(m)
        with pytest.raises(P.CartogramError) as e:
            c.iteration_gradient(m.values, 1.0, replay=True)
        assert e.value.code == P.CG_ESTATE
        with pytest.raises(P.CartogramError) as e:
            c.iteration_gradient(-m.values, 1.0)
        assert e.value.code == P.CG_EINVAL


def test_torch_autograd_function_gives_the_librarys_gradient():
    import torch
    m = synth.make_workload("voronoi16_64")
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="fp64") as c:
        c.set_map(m)
        ref_loss, ref_gv, ref_gb = c.iteration_gradient(m.values, 1.0, LAM)
        v = torch.tensor(m.values, dtype=torch.float64, requires_grad=True)
        b = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
        loss = P.iteration_loss(v, b, c, lam=LAM)
        loss.backward()
    assert abs(float(loss.detach()) - ref_loss) <= 1e-12 * abs(ref_loss)
    assert np.max(np.abs(v.grad.numpy() - ref_gv)) <= 1e-12 * np.max(np.abs(ref_gv))
    assert abs(float(b.grad) - ref_gb) <= 1e-12 * abs(ref_gb)


@pytest.mark.parametrize("K", [2, 3])
def test_gradient_through_several_iterations_matches_oracle_differences(orc, K):
    # through K outer iterations the rasteriser also depends on the vertices moved by the
    # earlier iterations; the FP64 reference is the central difference of the C oracle's
    # K-iteration loss with the same replayed schedules (the FP64 path records the same
    # schedules as the oracle's adaptive runs)
    from oracle import adjoint as adj
    m = synth.make_workload("voronoi16_64", L=32, n=8)
    blur, decay = 1.0, 0.5
    with P.Cartogram(m.Lx, m.Ly, blur, precision="fp64") as c:
        c.set_map(m)
        loss, gv, gb = c.iteration_gradient(m.values, blur, LAM, iterations=K)
    sch = adj.adaptive_schedules(orc, m, m.values, blur, decay, K)
    L_ref = adj.cartogram_loss(orc, m, m.values, blur, decay, sch, LAM)
    assert abs(loss - L_ref) < 1e-9 * abs(L_ref)

    def f(v, b):
        return adj.cartogram_loss(orc, m, v, b, decay, sch, LAM)

    # the loss is only piecewise smooth: the bilinear point map's derivative jumps where a
    # vertex moved by an earlier iteration crosses a grid-cell boundary, and a difference
    # step that straddles such a kink averages two one-sided slopes (at h = 1e-6 one region
    # of this map is off by 2e-6 that way); h = 1e-7 keeps every region on one side
    for i in range(m.n_regions):
        h = 1e-7 * m.values[i]
        vp, vm = m.values.copy(), m.values.copy()
        vp[i] += h
        vm[i] -= h
        fd = (f(vp, blur) - f(vm, blur)) / (2 * h)
        assert abs(fd - gv[i]) <= 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(gv))), (i, fd, gv[i])
    h = 1e-7
    fd = (f(m.values, blur + h) - f(m.values, blur - h)) / (2 * h)
    assert abs(fd - gb) <= 1e-6 * abs(fd), (fd, gb)


def test_gradient_through_several_iterations_against_gpu_differences():
    m = synth.make_workload("voronoi16_64")
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="fp64") as c:
        c.set_map(m)
        loss, gv, gb = c.iteration_gradient(m.values, 1.0, LAM, iterations=3, checkpoint=6)

        def f(v):
            return c.iteration_gradient(v, 1.0, LAM, replay=True, grad=False, iterations=3)

        # the loss is piecewise smooth (the point map's kinks, see above) and the GPU's loss
        # carries ~1e-13 of rounding from the rasteriser's atomic sums, which rules out steps
        # much below 1e-6; regions 5 and 11 of this map have a kink within 1e-6 of the point,
        # so the difference that stays on the point's own piece (central, forward or
        # backward) must match
        L0 = f(m.values)
        for i in (0, 5, 11):
            h = 1e-6 * m.values[i]
            vp, vm = m.values.copy(), m.values.copy()
            vp[i] += h
            vm[i] -= h
            Lp, Lm = f(vp), f(vm)
            diffs = [(Lp - Lm) / (2 * h), (Lp - L0) / h, (L0 - Lm) / h]
            err = min(abs(d - gv[i]) for d in diffs)
            assert err <= 1e-6 * abs(gv[i]), (i, diffs, gv[i])
        with pytest.raises(P.CartogramError) as e:
            c.iteration_gradient(m.values, 1.0, LAM, replay=True, iterations=2)  # recorded with 3
        assert e.value.code == P.CG_ESTATE
        assert np.array_equal(c.vertices(), m.xy) and c.history_length() == 0


@pytest.mark.parametrize("K", [1, 2])
def test_vjp_of_the_builtin_loss_gives_the_librarys_gradient(K):
    """The configured loss written in torch on the mapped vertices X' and areas A' (plus its
    direct dependence on the values through the target areas) gives, through the
    vector-Jacobian product, the gradient of cartogram_iteration_gradient."""
    import torch
    m = synth.make_workload("voronoi16_64")
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="fp64") as c:
        c.set_map(m)
        ref_loss, ref_gv, ref_gb = c.iteration_gradient(m.values, 1.0, LAM, iterations=K)
        X0 = torch.tensor(m.xy, dtype=torch.float64)
        v = torch.tensor(m.values, dtype=torch.float64, requires_grad=True)
        b = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
        xy, area = P.mapped_iterations(v, b, c, iterations=K)
        target = v * area.sum() / v.sum()
        loss = ((torch.log(area) - torch.log(target)) ** 2).sum() + LAM * ((xy - X0) ** 2).sum()
        loss.backward()
        assert np.array_equal(c.vertices(), m.xy) and c.history_length() == 0
    assert abs(float(loss.detach()) - ref_loss) <= 1e-12 * abs(ref_loss)
    assert np.max(np.abs(v.grad.numpy() - ref_gv)) <= 1e-11 * np.max(np.abs(ref_gv))
    assert abs(float(b.grad) - ref_gb) <= 1e-11 * abs(ref_gb)


def test_vjp_forward_is_the_mapped_map():
    # one iteration's X' and A' are the vertices and areas cartogram_integrate produces
    m = synth.make_workload("voronoi16_64")
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="fp64") as c:
        c.set_map(m)
        xy, area = c.iteration_vjp(m.values, 1.0, grad=False)
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="fp64", max_iter=1) as c:
        c.set_map(m)
        with pytest.raises(P.CartogramError):
            c.integrate()  # one iteration does not converge this map
        assert c.history_length() == 1
        assert np.max(np.abs(c.vertices() - xy)) < 1e-10
        err = c.area_errors()
    target = m.values * area.sum() / m.values.sum()
    assert np.max(np.abs((area / target - 1.0) - err)) < 1e-10


def test_vjp_of_another_loss_matches_central_differences():
    """A loss the library does not know: L = sum_i A'_i^2 / A0_i + sum_v w_v . X'_v with
    fixed weights w, against differences of the same loss with the schedule replayed."""
    m = synth.make_workload("voronoi16_64")
    rng = np.random.default_rng(7)
    w = rng.normal(size=(m.n_vertices, 2))
    with P.Cartogram(m.Lx, m.Ly, 1.0, precision="fp64") as c:
        c.set_map(m)
        xy, area = c.iteration_vjp(m.values, 1.0, iterations=2, grad=False)
        a0 = area.copy()

        def loss(v, b):
            x, a = c.iteration_vjp(v, b, iterations=2, replay=True, grad=False)
            return float(np.sum(a * a / a0) + np.sum(w * x))

        _, _, gv, gb = c.iteration_vjp(m.values, 1.0, iterations=2, replay=True, checkpoint=3,
                                       grad_xy=w, grad_area=2.0 * area / a0)
        L0 = loss(m.values, 1.0)
        for i in (0, 5, 11, 15):
            h = 1e-6 * m.values[i]
            vp, vm = m.values.copy(), m.values.copy()
            vp[i] += h
            vm[i] -= h
            Lp, Lm = loss(vp, 1.0), loss(vm, 1.0)
            diffs = [(Lp - Lm) / (2 * h), (Lp - L0) / h, (L0 - Lm) / h]
            assert min(abs(d - gv[i]) for d in diffs) <= 1e-5 * max(abs(gv[i]), 1e-3 * np.max(np.abs(gv))), \
                (i, diffs, gv[i])
        h = 1e-6
        Lp, Lm = loss(m.values, 1.0 + h), loss(m.values, 1.0 - h)
        diffs = [(Lp - Lm) / (2 * h), (Lp - L0) / h, (L0 - Lm) / h]
        assert min(abs(d - gb) for d in diffs) <= 1e-5 * abs(gb), (diffs, gb)
        # only dL/dA' given (dL/dX' = 0): the area part of the product alone
        _, _, gva, _ = c.iteration_vjp(m.values, 1.0, iterations=2, replay=True, grad_area=2.0 * area / a0)
        _, _, gvx, _ = c.iteration_vjp(m.values, 1.0, iterations=2, replay=True, grad_xy=w)
        assert np.max(np.abs(gva + gvx - gv)) <= 1e-12 * np.max(np.abs(gv))
