// Reverse-mode (adjoint) kernels of one outer iteration for a fixed step schedule, in
// FP64: the gradient of a loss on the mapped vertices and areas with respect to the
// regions' target values and the blur width.
//
// Forward of one iteration (the kernels of the FP64 path):
//   w_i = (V_i/A_i)(sum A/sum V) - 1;  rho' = sum_i w_i cov_i (exact coverage, edge pieces
//   + row prefix sums);  spec = W B(sigma) DCT-II(rho');  for every accepted step n of the
//   schedule, the fields v = -grad rho/rho at tau_n and tau_{n+1} (inverse passes) and
//   one predictor-corrector step of all grid points;  the vertices mapped through the
//   final grid;  the loss on their areas and displacements.
// The adjoint runs the steps backwards (positions recomputed from checkpoints), scatters
// the adjoint of every interpolated velocity into a field adjoint per time level,
// carries each level's field adjoint through v = -g/rho and the transposed transforms
// (DCT-II of the adjoint fields; the sine sums by the index-reversal identity
// sum_i x_i sin(pi m (i+1/2)/N) = DCT-II[(-1)^i x_i]_(N-m)) into a spectrum adjoint,
// and finally through the blur factor, the forward transform (an inverse-type cosine
// sum), the row prefix sums (suffix sums) and the edge pieces of the rasteriser.
#pragma once

#include "common.cuh"
#include "geometry.cuh"

namespace cg {

// Bilinear interpolation of a grid field at displacement (dx, dy) from cell centre
// (i, j), with the wall rule (the velocity kernel's interp_v), and what its adjoint
// needs: the four node indices and weights, the wall factors and the derivatives of
// the interpolated vector with respect to the position.
struct InterpD {
  int k[4];         // node indices (may repeat where clamped)
  double c[4];      // bilinear weights
  double sx, sy;    // wall factors of the x and y components
  double u[2];      // interpolated vector
  double du[2][2];  // du[comp][axis] = d u_comp / d position_axis
};

__device__ __forceinline__ void interp_d(const double2* __restrict__ v, int Lx, int Ly, int i, int j, double dx,
                                         double dy, InterpD& r) {
  const double flx = fmin(fmax(floor(dx), (double)(-2 - Lx)), (double)(Lx + 2));
  const double fly = fmin(fmax(floor(dy), (double)(-2 - Ly)), (double)(Ly + 2));
  const int ix = i + (int)flx, iy = j + (int)fly;
  const double fx = dx - flx, fy = dy - fly;
  const int i0 = min(max(ix, 0), Lx - 1), i1 = min(max(ix + 1, 0), Lx - 1);
  const int j0 = min(max(iy, 0), Ly - 1), j1 = min(max(iy + 1, 0), Ly - 1);
  r.k[0] = j0 * Lx + i0;
  r.k[1] = j0 * Lx + i1;
  r.k[2] = j1 * Lx + i0;
  r.k[3] = j1 * Lx + i1;
  const double2 a = v[r.k[0]], b = v[r.k[1]], c = v[r.k[2]], d = v[r.k[3]];
  const double gx = 1.0 - fx, gy = 1.0 - fy;
  r.c[0] = gx * gy;
  r.c[1] = fx * gy;
  r.c[2] = gx * fy;
  r.c[3] = fx * fy;
  const double ux = gy * (gx * a.x + fx * b.x) + fy * (gx * c.x + fx * d.x);
  const double uy = gy * (gx * a.y + fx * b.y) + fy * (gx * c.y + fx * d.y);
  // raw derivatives along x (weights' fx) and y (weights' fy)
  double dux_dx = gy * (b.x - a.x) + fy * (d.x - c.x), dux_dy = (gx * c.x + fx * d.x) - (gx * a.x + fx * b.x);
  double duy_dx = gy * (b.y - a.y) + fy * (d.y - c.y), duy_dy = (gx * c.y + fx * d.y) - (gx * a.y + fx * b.y);
  // wall factors min(1, 2x, 2(L - x)) inside the half-cell bands (i0 == i1 there, so the
  // raw value does not depend on the position along that axis)
  r.sx = 1.0;
  r.sy = 1.0;
  double dsx = 0.0, dsy = 0.0;
  if (ix < 0 || ix >= Lx - 1) {
    const double x = (double)i + 0.5 + dx;
    const double m1 = 2.0 * x, m2 = 2.0 * ((double)Lx - x);
    if (m1 < 1.0 && m1 <= m2) {
      r.sx = m1;
      dsx = 2.0;
    } else if (m2 < 1.0) {
      r.sx = m2;
      dsx = -2.0;
    }
  }
  if (iy < 0 || iy >= Ly - 1) {
    const double y = (double)j + 0.5 + dy;
    const double m1 = 2.0 * y, m2 = 2.0 * ((double)Ly - y);
    if (m1 < 1.0 && m1 <= m2) {
      r.sy = m1;
      dsy = 2.0;
    } else if (m2 < 1.0) {
      r.sy = m2;
      dsy = -2.0;
    }
  }
  r.u[0] = ux * r.sx;
  r.u[1] = uy * r.sy;
  r.du[0][0] = dux_dx * r.sx + ux * dsx;
  r.du[0][1] = dux_dy * r.sx;
  r.du[1][0] = duy_dx * r.sy;
  r.du[1][1] = duy_dy * r.sy + uy * dsy;
}

// Scatter the adjoint g of an interpolated vector into the field adjoint L ([N][2]).
__device__ __forceinline__ void scatter_field(const InterpD& r, double gx, double gy, double* L) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    atomicAdd(L + 2 * r.k[q], r.c[q] * r.sx * gx);
    atomicAdd(L + 2 * r.k[q] + 1, r.c[q] * r.sy * gy);
  }
}

__device__ __forceinline__ double clamp_mask(double v, double lo, double hi) {
  return (v < lo || v > hi) ? 0.0 : 1.0;
}

// Adjoint of one predictor-corrector step of every grid point (the step kernel's
// arithmetic: u0 at the position, clamped predictor, u1 there, clamped corrector).
// lam: adjoint of the displacements after the step on entry, before it on exit.
__global__ void heun_adjoint_kernel(const double2* __restrict__ d, const double2* __restrict__ v0,
                                    const double2* __restrict__ v1, double h, double2* lam, double* L0,
                                    double* L1, int Lx, int Ly, int log2Lx) {
  const int N = Lx * Ly;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const int i = p & (Lx - 1), j = p >> log2Lx;
    const double lox = -((double)i + 0.5), hix = (double)(Lx - i) - 0.5;
    const double loy = -((double)j + 0.5), hiy = (double)(Ly - j) - 0.5;
    const double2 dd = d[p];
    InterpD a, b;
    interp_d(v0, Lx, Ly, i, j, dd.x, dd.y, a);
    const double prx = dd.x + h * a.u[0], pry = dd.y + h * a.u[1];
    const double px = fmin(fmax(prx, lox), hix), py = fmin(fmax(pry, loy), hiy);
    interp_d(v1, Lx, Ly, i, j, px, py, b);
    const double crx = dd.x + 0.5 * h * (a.u[0] + b.u[0]), cry = dd.y + 0.5 * h * (a.u[1] + b.u[1]);
    const double2 lc = lam[p];
    const double gx = lc.x * clamp_mask(crx, lox, hix), gy = lc.y * clamp_mask(cry, loy, hiy);
    // corrector: c = d + h/2 (u0 + u1)
    double ldx = gx, ldy = gy;
    double lu0x = 0.5 * h * gx, lu0y = 0.5 * h * gy;
    const double lu1x = 0.5 * h * gx, lu1y = 0.5 * h * gy;
    // u1 = interp(v1, p)
    scatter_field(b, lu1x, lu1y, L1);
    const double lpx = (b.du[0][0] * lu1x + b.du[1][0] * lu1y) * clamp_mask(prx, lox, hix);
    const double lpy = (b.du[0][1] * lu1x + b.du[1][1] * lu1y) * clamp_mask(pry, loy, hiy);
    // predictor: p = d + h u0
    ldx += lpx;
    ldy += lpy;
    lu0x += h * lpx;
    lu0y += h * lpy;
    // u0 = interp(v0, d)
    scatter_field(a, lu0x, lu0y, L0);
    ldx += a.du[0][0] * lu0x + a.du[1][0] * lu0y;
    ldy += a.du[0][1] * lu0x + a.du[1][1] * lu0y;
    lam[p] = make_double2(ldx, ldy);
  }
}

// Field adjoint of one time level -> adjoints of rho and of the two gradient components
// (v = -g/rho: d v/d g = -1/rho, d v/d rho = -v/rho), the gradient components sign-flipped
// by (-1)^i and (-1)^j for the sine sums.
__global__ void node_adjoint_kernel(const double* __restrict__ L, const double2* __restrict__ v,
                                    const double* __restrict__ rho, double* a_rho, double* a_gx, double* a_gy,
                                    int Lx, int N) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const int i = p % Lx, j = p / Lx;
    const double lx = L[2 * p], ly = L[2 * p + 1];
    const double r = rho[p];
    const double2 vv = v[p];
    a_rho[p] = -(lx * vv.x + ly * vv.y) / r;
    a_gx[p] = (i & 1) ? lx / r : -lx / r;
    a_gy[p] = (j & 1) ? ly / r : -ly / r;
  }
}

// lam_spec[n][m] += f(tau)/(Lx Ly) (Crho + (-pi m/Lx) Cx[n][Lx-m] + (-pi n/Ly) Cy[Ly-n][m]),
// from the DCT-II outputs of the three adjoint fields (each holding the weights
// (1 + (m>0))(1 + (n>0)), which are divided out). f is the damping of the inverse
// pass: exp(-pi^2 tau m^2/Lx^2) exp(-pi^2 tau n^2/Ly^2).
// The damping and the wavenumber factors are separable: a block evaluates those of the
// columns once into shared memory (Lx <= 1024) and one of each per row, so a coefficient
// costs no exponential and no division (GB300's FP64 rate makes both expensive); the
// weights' divisions are by powers of two, so their products are the same numbers.
__global__ void spec_accumulate_kernel(const double* __restrict__ Crho, const double* __restrict__ Cx,
                                       const double* __restrict__ Cy, double* lam_spec, double tau, int Lx,
                                       int Ly) {
  __shared__ double fxm[1024], gxm[1024];
  const double kx = kPi * kPi * tau / ((double)Lx * Lx), ky = kPi * kPi * tau / ((double)Ly * Ly);
  for (int m = threadIdx.x; m < Lx; m += blockDim.x) {
    fxm[m] = exp(-kx * m * m) / Lx;
    gxm[m] = -kPi * m / Lx;
  }
  __syncthreads();
  for (int n = blockIdx.x; n < Ly; n += gridDim.x) {
    const double fyn = exp(-ky * n * n) / Ly, gyn = -kPi * n / Ly;
    const double wn = n == 0 ? 1.0 : 2.0;
    const double* crow = Crho + (size_t)n * Lx;
    const double* xrow = Cx + (size_t)n * Lx;
    const double* yrow = Cy + (size_t)(Ly - n) * Lx;  // read only for n > 0
    double* out = lam_spec + (size_t)n * Lx;
    for (int m = threadIdx.x; m < Lx; m += blockDim.x) {
      if (m == 0 && n == 0) continue;
      const double wm = m == 0 ? 1.0 : 2.0;
      double s = crow[m] * (1.0 / (wm * wn));
      if (m > 0) s += gxm[m] * xrow[Lx - m] * (1.0 / (2.0 * wn));
      if (n > 0) s += gyn * yrow[m] * (1.0 / (wm * 2.0));
      out[m] += (fxm[m] * fyn) * s;
    }
  }
}

// d L/d sigma_k = sum_mn lam_spec spec (-sigma_k) ((pi m/Lx)^2 + (pi n/Ly)^2), and the
// input of the density adjoint: lam_spec W B (Lx Ly) (an inverse pass then gives
// sum_mn lam_spec W B cos cos).
__global__ void spec_tail_kernel(const double* __restrict__ lam_spec, const double* __restrict__ spec,
                                 const double* __restrict__ bx, const double* __restrict__ by, double sigma,
                                 double* specp, double* dsigma, int Lx, int Ly) {
  __shared__ double red[256];
  const int N = Lx * Ly;
  double acc = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const int m = p % Lx, n = p / Lx;
    if (m == 0 && n == 0) {
      specp[p] = 0.0;
      continue;
    }
    const double km = kPi * m / Lx, kn = kPi * n / Ly;
    acc += lam_spec[p] * spec[p] * (-sigma) * (km * km + kn * kn);
    const double w = (m == 0 ? 1.0 : 2.0) * (n == 0 ? 1.0 : 2.0);
    specp[p] = lam_spec[p] * w * bx[m] * by[n] * ((double)Lx * Ly);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(dsigma, red[0]);
}

// In-place inclusive suffix sum of every row (the adjoint of the row prefix sums).
__global__ void row_suffix_kernel(double* __restrict__ acc, int Lx) {
  if (threadIdx.x != 0) return;
  double* row = acc + (size_t)blockIdx.x * Lx;
  double s = 0.0;
  for (int i = Lx - 1; i >= 0; --i) {
    s += row[i];
    row[i] = s;
  }
}

// Adjoint of the edge pieces: d L/d w_r += sum over the pieces of region r's edges of
// the piece's deposits weighted by the (suffix-summed) density adjoint.
__global__ void raster_adjoint_kernel(const double2* __restrict__ xy, const int* __restrict__ next,
                                      const int* __restrict__ vreg, const double* __restrict__ lam, double* grad_w,
                                      int Lx, int Ly, int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const double2 P = xy[v], Q = xy[next[v]];
    if (Q.y - P.y == 0.0) continue;
    double g = 0.0;
    edge_pieces(P, Q, Lx, Ly, [&](double ax, double ay, double bx, double by, double, double, int ii, int jj) {
      const double pdy = by - ay;
      if (pdy == 0.0 || jj < 0 || jj >= Ly) return;
      const double mx = 0.5 * (ax + bx);
      const double c = -pdy;
      const double* row = lam + (size_t)jj * Lx;
      if (ii < 0) {
        g += c * row[0];
      } else if (ii < Lx) {
        g += c * ((double)(ii + 1) - mx) * row[ii];
        if (ii + 1 < Lx) g += c * (mx - (double)ii) * row[ii + 1];
      }
    });
    atomicAdd(grad_w + vreg[v], g);
  }
}

// d L/d X'_v for every vertex of the mapped rings: the area adjoint of its region times
// the shoelace derivative (half the difference of its neighbours' coordinates), plus the
// displacement penalty 2 lam (X'_v - X_v).
__global__ void vertex_adjoint_kernel(const double2* __restrict__ xy1, const double2* __restrict__ xy0,
                                      const int* __restrict__ next, const int* __restrict__ prev,
                                      const int* __restrict__ vreg, const double* __restrict__ dLdA, double lam,
                                      double2* g, int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const double2 a = xy1[next[v]], b = xy1[prev[v]], x1 = xy1[v], x0 = xy0[v];
    const double gA = dLdA[vreg[v]];
    g[v] = make_double2(gA * 0.5 * (a.y - b.y) + 2.0 * lam * (x1.x - x0.x),
                        gA * 0.5 * (b.x - a.x) + 2.0 * lam * (x1.y - x0.y));
  }
}

// Adjoint of mapping the (fixed) vertices through the grid: their adjoints scattered
// into the grid displacements' adjoint with the map's bilinear weights.
__global__ void map_adjoint_kernel(const double2* __restrict__ xy0, const double2* __restrict__ g, double* lamD,
                                   int Lx, int Ly, int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const double2 q = xy0[v];
    const double u = q.x - 0.5, w = q.y - 0.5;
    int i0 = (int)floor(u), j0 = (int)floor(w);
    i0 = i0 < 0 ? 0 : (i0 > Lx - 2 ? Lx - 2 : i0);
    j0 = j0 < 0 ? 0 : (j0 > Ly - 2 ? Ly - 2 : j0);
    const double fx = u - i0, fy = w - j0;
    const size_t k = (size_t)j0 * Lx + i0;
    const double c[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
    const size_t kk[4] = {k, k + 1, k + Lx, k + Lx + 1};
    const double2 gg = g[v];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      atomicAdd(lamD + 2 * kk[t], c[t] * gg.x);
      atomicAdd(lamD + 2 * kk[t] + 1, c[t] * gg.y);
    }
  }
}

// ---- vertex adjoints (gradients through several outer iterations) -----------------

// Adjoint of the exact coverage with respect to the ring vertices: moving an edge sweeps
// area across its outward normal (d.y, -d.x)/|d| of a counter-clockwise ring, so
// d/dP sum_c lam_c w_r cov_r(c) = w_r sum over the edge's pieces of lam_c (d.y, -d.x)
// times the integral of the hat function of P (1 - s) over the piece, and likewise for
// Q with s. lam is the density adjoint per cell (before the suffix sums).
__global__ void coverage_vertex_adjoint_kernel(const double2* __restrict__ xy, const int* __restrict__ next,
                                               const int* __restrict__ vreg, const double* __restrict__ w,
                                               const double* __restrict__ lam, double* g, int Lx, int Ly, int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const double2 P = xy[v], Q = xy[next[v]];
    const double dx = Q.x - P.x, dy = Q.y - P.y;
    if (dx == 0.0 && dy == 0.0) continue;
    const double wr = w[vreg[v]];
    double aP = 0.0, aQ = 0.0;  // sum of lam_c times the hat integrals
    edge_pieces(P, Q, Lx, Ly, [&](double, double, double, double, double s0, double s1, int ii, int jj) {
      if (jj < 0 || jj >= Ly || ii < 0 || ii >= Lx) return;
      const double lc = lam[(size_t)jj * Lx + ii];
      const double q = 0.5 * (s1 * s1 - s0 * s0);
      aP += lc * ((s1 - s0) - q);
      aQ += lc * q;
    });
    const double nx = wr * dy, ny = -wr * dx;
    atomicAdd(g + 2 * v, aP * nx);
    atomicAdd(g + 2 * v + 1, aP * ny);
    atomicAdd(g + 2 * next[v], aQ * nx);
    atomicAdd(g + 2 * next[v] + 1, aQ * ny);
  }
}

// Vertex adjoint through the map X' = X + (bilinear interpolation of the grid
// displacements D at X): lam_out = lam + (d D(X)/d X)^T lam.
__global__ void map_jacobian_adjoint_kernel(const double2* __restrict__ xy, const double2* __restrict__ D,
                                            const double2* __restrict__ lam, double2* lam_out, int Lx, int Ly,
                                            int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const double2 q = xy[v];
    const double u = q.x - 0.5, wv = q.y - 0.5;
    int i0 = (int)floor(u), j0 = (int)floor(wv);
    i0 = i0 < 0 ? 0 : (i0 > Lx - 2 ? Lx - 2 : i0);
    j0 = j0 < 0 ? 0 : (j0 > Ly - 2 ? Ly - 2 : j0);
    const double fx = u - i0, fy = wv - j0;
    const size_t k = (size_t)j0 * Lx + i0;
    const double2 a = D[k], b = D[k + 1], c = D[k + Lx], d = D[k + Lx + 1];
    const double dxx = (1 - fy) * (b.x - a.x) + fy * (d.x - c.x);  // d Dx / dx
    const double dyx = (1 - fy) * (b.y - a.y) + fy * (d.y - c.y);  // d Dy / dx
    const double dxy = (1 - fx) * (c.x - a.x) + fx * (d.x - b.x);  // d Dx / dy
    const double dyy = (1 - fx) * (c.y - a.y) + fx * (d.y - b.y);  // d Dy / dy
    const double2 l = lam[v];
    lam_out[v] = make_double2(l.x + l.x * dxx + l.y * dyx, l.y + l.x * dxy + l.y * dyy);
  }
}

// g[v] += dL/dA_(region of v) times the shoelace derivative of the region's area.
__global__ void shoelace_adjoint_kernel(const double2* __restrict__ xy, const int* __restrict__ next,
                                        const int* __restrict__ prev, const int* __restrict__ vreg,
                                        const double* __restrict__ dLdA, double2* g, int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const double2 a = xy[next[v]], b = xy[prev[v]];
    const double gA = dLdA[vreg[v]];
    double2 t = g[v];
    t.x += gA * 0.5 * (a.y - b.y);
    t.y += gA * 0.5 * (b.x - a.x);
    g[v] = t;
  }
}

}  // namespace cg
