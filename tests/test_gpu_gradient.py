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
    assert abs(float(loss) - ref_loss) <= 1e-12 * abs(ref_loss)
    assert np.max(np.abs(v.grad.numpy() - ref_gv)) <= 1e-12 * np.max(np.abs(ref_gv))
    assert abs(float(b.grad) - ref_gb) <= 1e-12 * abs(ref_gb)
