"""FP64 reverse-mode reference for the gradient of one outer iteration's loss.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): plain PyTorch CPU float64 with
autograd, written from the paper's equations, independent of the CUDA path.

One outer iteration (main text, section on benchmarking: rasterise, blur, integrate,
map) as a differentiable function of the regions' target values V and the blur width
sigma, for a FIXED step schedule (the accepted step sizes of an adaptive run: the
accept/reject decisions and the step sizes are held constant, so the function is
smooth in V and sigma):
  w_i   = (V_i / A_i) (sum A / sum V) - 1                 region density / mean - 1
  rho'  = sum_i w_i cov_i                                  exact coverage (orc_coverage)
  spec  = W B(sigma) DCT-II(rho'),  spec_00 = 0            SI Eq. rhotilde_mn, blur factor
  rho(t), grad rho(t) from spec damped by f(t)             SI Eqs. rhoxyt, fmn_diff (D = 1)
  v     = -grad rho / rho at the grid points               Fick's law
  Heun steps of all grid points with the lattice-with-walls interpolation and the
  clamping of the oracle's orc_heun_step
  X'    = the input vertices mapped through the final grid (orc_map_points)
  L     = sum_i (ln A'_i - ln A^_i)^2 + lam sum_v |X'_v - X_v|^2,  A^_i = V_i sum A' / sum V
The forward is pinned to the C oracle's integration (identical positions for the same
schedule); autograd gives the exact derivative of this forward.
"""
import math

import numpy as np
import torch

PI = math.pi
_T = torch.float64


def _cos(L):
    m = torch.arange(L, dtype=_T)[:, None]
    i = torch.arange(L, dtype=_T)[None, :]
    return torch.cos(PI * m * (i + 0.5) / L)  # [m, i]


def _sin(L):
    m = torch.arange(L, dtype=_T)[:, None]
    i = torch.arange(L, dtype=_T)[None, :]
    return torch.sin(PI * m * (i + 0.5) / L)


def _lattice(x, L):
    """Interpolation cell a, its ends and the weight along one axis (lattice
    {0, 1/2, 3/2, ..., L-1/2, L}: walls plus cell centres)."""
    a = torch.where(x < 0.5, torch.zeros_like(x), torch.where(x >= L - 0.5, torch.full_like(x, L),
                                                               torch.floor(x.detach() - 0.5) + 1)).long()

    def pos(k):
        return torch.where(k == 0, torch.zeros_like(x), torch.where(k == L + 1, torch.full_like(x, L), k.to(_T) - 0.5))

    xa, xb = pos(a), pos(a + 1)
    return a, (x - xa) / (xb - xa)


def _interp(vx, vy, x, y):
    Ly, Lx = vx.shape
    a, wx = _lattice(x, Lx)
    b, wy = _lattice(y, Ly)

    def value(aa, bb):
        ghost_x = (aa == 0) | (aa == Lx + 1)
        ghost_y = (bb == 0) | (bb == Ly + 1)
        ia = torch.clamp(aa - 1, 0, Lx - 1)
        jb = torch.clamp(bb - 1, 0, Ly - 1)
        ox = torch.where(ghost_x, torch.zeros_like(x), vx[jb, ia])
        oy = torch.where(ghost_y, torch.zeros_like(y), vy[jb, ia])
        return ox, oy

    v00, v10, v01, v11 = value(a, b), value(a + 1, b), value(a, b + 1), value(a + 1, b + 1)
    c00, c10, c01, c11 = (1 - wx) * (1 - wy), wx * (1 - wy), (1 - wx) * wy, wx * wy
    return (c00 * v00[0] + c10 * v10[0] + c01 * v01[0] + c11 * v11[0],
            c00 * v00[1] + c10 * v10[1] + c01 * v01[1] + c11 * v11[1])


def _map_points(X, Y, px, py):
    Ly, Lx = X.shape
    u, w = px - 0.5, py - 0.5
    i0 = torch.clamp(torch.floor(u.detach()), 0, Lx - 2).long()
    j0 = torch.clamp(torch.floor(w.detach()), 0, Ly - 2).long()
    fx, fy = u - i0, w - j0
    c00, c10, c01, c11 = (1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy
    ox = c00 * X[j0, i0] + c10 * X[j0, i0 + 1] + c01 * X[j0 + 1, i0] + c11 * X[j0 + 1, i0 + 1]
    oy = c00 * Y[j0, i0] + c10 * Y[j0, i0 + 1] + c01 * Y[j0 + 1, i0] + c11 * Y[j0 + 1, i0 + 1]
    return ox, oy


def _region_areas(m, x, y):
    areas = torch.zeros(m.n_regions, dtype=_T)
    for k in range(m.n_rings):
        a, b = int(m.ring_offsets[k]), int(m.ring_offsets[k + 1])
        xs, ys = x[a:b], y[a:b]
        ring = 0.5 * torch.sum(xs * torch.roll(ys, -1) - torch.roll(xs, -1) * ys)
        areas = areas.index_add(0, torch.tensor([int(m.ring_region[k])]), ring.reshape(1))
    return areas


class Iteration:
    """Precomputed constants of one outer iteration on map m (geometry fixed)."""

    def __init__(self, m, cov, A):
        self.m = m
        self.Lx, self.Ly = m.Lx, m.Ly
        self.cov = torch.as_tensor(cov, dtype=_T)
        self.A = torch.as_tensor(A, dtype=_T)
        self.Cx, self.Cy = _cos(self.Lx), _cos(self.Ly)
        self.Sx, self.Sy = _sin(self.Lx), _sin(self.Ly)
        mm = torch.arange(self.Lx, dtype=_T)[None, :]
        nn = torch.arange(self.Ly, dtype=_T)[:, None]
        self.mm, self.nn = mm, nn
        self.W = torch.where(mm == 0, 1.0, 2.0) * torch.where(nn == 0, 1.0, 2.0)
        self.x0 = torch.as_tensor(m.xy[:, 0], dtype=_T)
        self.y0 = torch.as_tensor(m.xy[:, 1], dtype=_T)

    def spectrum(self, values, blur):
        w = values / self.A * (self.A.sum() / values.sum()) - 1.0
        rho_p = torch.tensordot(w, self.cov, 1)  # [Ly, Lx]
        raw = self.Cy @ rho_p @ self.Cx.T  # [n, m]
        kx = PI * self.mm / self.Lx
        ky = PI * self.nn / self.Ly
        B = torch.exp(-0.5 * kx * kx * blur * blur) * torch.exp(-0.5 * ky * ky * blur * blur)
        spec = self.W * B * raw
        mask = torch.ones_like(spec)
        mask[0, 0] = 0.0
        return spec * mask

    def velocity(self, spec, tau):
        f = torch.exp(-PI * PI * tau * self.mm ** 2 / self.Lx ** 2) * torch.exp(-PI * PI * tau * self.nn ** 2 / self.Ly ** 2)
        s = spec * f / (self.Lx * self.Ly)
        rho = 1.0 + self.Cy.T @ s @ self.Cx
        gx = self.Cy.T @ (s * (-PI * self.mm / self.Lx)) @ self.Sx
        gy = self.Sy.T @ (s * (-PI * self.nn / self.Ly)) @ self.Cx
        return -gx / rho, -gy / rho

    def integrate(self, spec, steps):
        """Heun steps of all grid points with the given accepted step sizes."""
        Lx, Ly = self.Lx, self.Ly
        X = (torch.arange(Lx, dtype=_T)[None, :] + 0.5).expand(Ly, Lx).reshape(-1)
        Y = (torch.arange(Ly, dtype=_T)[:, None] + 0.5).expand(Ly, Lx).reshape(-1)
        tau = 0.0
        v0 = self.velocity(spec, tau)
        for h in steps:
            v1 = self.velocity(spec, tau + h)
            ax, ay = _interp(v0[0], v0[1], X, Y)
            px = torch.clamp(X + h * ax, 0.0, Lx)
            py = torch.clamp(Y + h * ay, 0.0, Ly)
            bx, by = _interp(v1[0], v1[1], px, py)
            X = torch.clamp(X + 0.5 * h * (ax + bx), 0.0, Lx)
            Y = torch.clamp(Y + 0.5 * h * (ay + by), 0.0, Ly)
            tau = tau + h
            v0 = v1
        return X.reshape(Ly, Lx), Y.reshape(Ly, Lx)

    def loss(self, values, blur, steps, lam):
        spec = self.spectrum(values, blur)
        X, Y = self.integrate(spec, steps)
        x1, y1 = _map_points(X, Y, self.x0, self.y0)
        A1 = _region_areas(self.m, x1, y1)
        target = values * A1.sum() / values.sum()
        r = torch.log(A1) - torch.log(target)
        return torch.sum(r * r) + lam * torch.sum((x1 - self.x0) ** 2 + (y1 - self.y0) ** 2), (X, Y)


def accepted_steps(sched_h, sched_acc):
    """Accepted step sizes, in order, from an adaptive run's attempt record."""
    return [float(h) for h, a in zip(sched_h, sched_acc) if a]


def gradient(it: Iteration, values, blur, steps, lam):
    """Loss and its FP64 gradient with respect to the values and the blur width."""
    v = torch.tensor(np.asarray(values, dtype=np.float64), requires_grad=True)
    s = torch.tensor(float(blur), dtype=_T, requires_grad=True)
    L, _ = it.loss(v, s, steps, lam)
    L.backward()
    return float(L.detach()), v.grad.numpy().copy(), float(s.grad)


def adaptive_schedules(orc, m, values, blur, decay, K):
    """The accepted step sizes of K adaptive outer iterations with the C oracle (the
    schedule that the FP64 GPU path records too)."""
    xy = np.array(m.xy, dtype=np.float64)
    out = []
    for k in range(K):
        A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, xy)
        rho = orc.rasterize(m.Lx, m.Ly, values, A, m.ring_offsets, m.ring_region, xy) / (np.sum(values) / A.sum())
        r = orc.integrate(orc.forward(rho, blur * decay ** k))
        out.append(accepted_steps(r.sched_h, r.sched_acc))
        xy = orc.map_points(r.X, r.Y, xy)
    return out


def cartogram_loss(orc, m, values, blur, decay, schedules, lam):
    """The loss after len(schedules) outer iterations of the C oracle with those fixed step
    schedules (rasterisation, blurred transform, replayed integration, point map), in FP64;
    its central differences give the FP64 reference gradient through several iterations
    (where the rasteriser's dependence on the moved vertices enters)."""
    values = np.asarray(values, dtype=np.float64)
    xy = np.array(m.xy, dtype=np.float64)
    for k, steps in enumerate(schedules):
        A = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, xy)
        rho = orc.rasterize(m.Lx, m.Ly, values, A, m.ring_offsets, m.ring_region, xy) / (values.sum() / A.sum())
        X, Y = orc.integrate_replay(orc.forward(rho, blur * decay ** k), steps)
        xy = orc.map_points(X, Y, xy)
    A1 = orc.region_areas(m.n_regions, m.ring_offsets, m.ring_region, xy)
    r = np.log(A1) - np.log(values * A1.sum() / values.sum())
    return float(np.sum(r * r) + lam * np.sum((xy - m.xy) ** 2))
