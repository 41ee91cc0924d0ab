// The paper's linear-equalisation flow (SI Eq. fmn_fast: f_mn = 1 - t for t <= 1).
//
// Its flux is constant in time: with f'_mn = -1, SI Eqs. Jxmn and Jymn give
// J = -grad Phi with Phi~_mn = rho~_mn / (pi^2 (m^2/Lx^2 + n^2/Ly^2)), evaluated once per
// integration by the inverse transform passes. The density is rho(t) = (1-t) rho0 + t
// rho_bar (main text Eq. rho_ffb, rho_bar = 1 here), so v(t) = J / rho(t) needs no
// transform per step: the step kernel forms v at the four grid points around each
// position from J and rho0 and interpolates (the paper computes v at the grid points
// with basic arithmetic and interpolates between them). The integration ends at t = 1.
#pragma once

#include "advect.cuh"

namespace cg {

// Phi~ = rho~ / (pi^2 k^2), Phi~_00 = 0, from the FP64 spectrum.
template <typename T>
__global__ void phi_spectrum_kernel(const double* __restrict__ spec, T* __restrict__ phi, int Lx, int Ly) {
  const int N = Lx * Ly;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const int m = p % Lx, n = p / Lx;
    const double k2 = (double)m * m / ((double)Lx * Lx) + (double)n * n / ((double)Ly * Ly);
    phi[p] = p == 0 ? T(0) : (T)(spec[p] / (kPi * kPi * k2));
  }
}

// v(t) at a grid node from the flux and the initial density.
template <typename T>
__device__ __forceinline__ V2<T> node_v(V2<T> J, T rho0, T t) {
  const T inv = T(1) / ((T(1) - t) * rho0 + t);
  return mk2<T>(J.x * inv, J.y * inv);
}

// Bilinear interpolation of v(t) = J / rho(t) between the grid points, with the same
// clamped lattice and wall rule as the diffusion flow.
template <typename T>
__device__ __forceinline__ V2<T> interp_lin(const V2<T>* __restrict__ J, const T* __restrict__ rho0, T t,
                                            int Lx, int Ly, int i, int j, T dx, T dy) {
  const T flx = min(max(floor(dx), T(-2 - Lx)), T(Lx + 2));
  const T fly = min(max(floor(dy), T(-2 - Ly)), T(Ly + 2));
  const int ix = i + (int)flx, iy = j + (int)fly;
  const T fx = dx - flx, fy = dy - fly;
  const int i0 = min(max(ix, 0), Lx - 1), i1 = min(max(ix + 1, 0), Lx - 1);
  const int j0 = min(max(iy, 0), Ly - 1), j1 = min(max(iy + 1, 0), Ly - 1);
  const int r0 = j0 * Lx, r1 = j1 * Lx;
  const V2<T> a = node_v(J[r0 + i0], rho0[r0 + i0], t), b = node_v(J[r0 + i1], rho0[r0 + i1], t);
  const V2<T> c = node_v(J[r1 + i0], rho0[r1 + i0], t), d = node_v(J[r1 + i1], rho0[r1 + i1], t);
  const T gx = T(1) - fx, gy = T(1) - fy;
  T ux = gy * (gx * a.x + fx * b.x) + fy * (gx * c.x + fx * d.x);
  T uy = gy * (gx * a.y + fx * b.y) + fy * (gx * c.y + fx * d.y);
  const T x = (T)i + T(0.5) + dx, y = (T)j + T(0.5) + dy;
  if (ix < 0 || ix >= Lx - 1) ux *= min(T(1), min(T(2) * x, T(2) * ((T)Lx - x)));
  if (iy < 0 || iy >= Ly - 1) uy *= min(T(1), min(T(2) * y, T(2) * ((T)Ly - y)));
  return mk2<T>(ux, uy);
}

// End of the attempted step t -> t1 (the step reaching t = 1 ends exactly there).
__device__ __forceinline__ double linear_t1(double t, double h) { return (t + h >= 1.0) ? 1.0 : t + h; }

// Controller of the linear flow: accept / reject, next step capped by cfl / max|v| and by
// 1 - t; done once an accepted step reaches t = 1.
__device__ __forceinline__ void control_linear(DevState* st, const StepParams& sp,
                                               cudaGraphConditionalHandle handle, int use_cond) {
  const double e = sqrt(__longlong_as_double((long long)st->err2_bits));
  const double vmax_new = sqrt(__longlong_as_double((long long)st->vmax2_bits));
  int status = kRunning;
  double h = st->h;
  if (st->bad) {
    status = kStepFail;
  } else if (e <= sp.atol) {
    st->parity ^= 1;
    st->t = linear_t1(st->t, h);
    st->accepted += 1;
    st->vmax = vmax_new;
    if (st->t >= 1.0) status = kDone;
    else h *= sp.grow;
  } else {
    st->rejected += 1;
    h *= sp.shrink;
  }
  if (status == kRunning) {
    if (st->accepted + st->rejected >= sp.max_steps || !(h > sp.h_min)) status = kStepFail;
    else {
      if (st->vmax > 0.0 && h * st->vmax > sp.cfl) h = sp.cfl / st->vmax;
      if (h > 1.0 - st->t) h = 1.0 - st->t;
    }
  }
  st->h = h;
  st->status = status;
  st->err2_bits = 0;
  st->vmax2_bits = 0;
  st->dev_bits = 0;
  st->ticket = 0;
  st->bad = 0;
  if (status != kRunning && use_cond) cudaGraphSetConditional(handle, 0);
}

// One attempted step of the linear flow for all grid points (two per thread), plus the
// maximum of |v(t1)| over the grid nodes this thread owns; the last block runs the
// controller. Step mode only (buffers by parity).
template <typename T>
__global__ void __launch_bounds__(256) linear_step_kernel(DevState* st, StepParams sp, const V2<T>* J,
                                                          const T* rho0, V2<T>* dbuf0, V2<T>* dbuf1, int Lx,
                                                          int Ly, int log2Lx,
                                                          cudaGraphConditionalHandle handle,
                                                          int use_cond, unsigned int max_body) {
  __shared__ unsigned long long s_err2, s_v2;
  __shared__ unsigned int s_warps;
  if (threadIdx.x == 0) {
    s_err2 = 0ull;
    s_v2 = 0ull;
    s_warps = 0u;
  }
  __syncthreads();
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (blockIdx.x == 0 && threadIdx.x == 0 && use_cond && atomicAdd(&st->body_iters, 1u) + 1u > max_body)
    cudaGraphSetConditional(handle, 0);  // termination guard; the status stays short of done
  if (st->status != kRunning) {
    // an attempt after the end of the integration (unrolled graph body): keep the loop
    // from running on
    if (blockIdx.x == 0 && threadIdx.x == 0 && use_cond) cudaGraphSetConditional(handle, 0);
    return;
  }
  const int par = st->parity;
  const V2<T>* din = par ? dbuf1 : dbuf0;
  V2<T>* dout = par ? dbuf0 : dbuf1;
  const double t0d = st->t, t1d = linear_t1(t0d, st->h);
  const T t0 = (T)t0d, t1 = (T)t1d, h = (T)(t1d - t0d), hh = (T)(0.5 * (t1d - t0d));
  const int npairs = (Lx * Ly) >> 1;
  T e2 = T(0), v2 = T(0);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += gridDim.x * blockDim.x) {
    const int p = 2 * q;
    const int i = p & (Lx - 1), j = p >> log2Lx;
    V2<T> d[2];
    load_pair(din + p, d);
    V2<T> o[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int ik = i + k;
      const T lox = -((T)ik + T(0.5)), hix = (T)(Lx - ik) - T(0.5);
      const T loy = -((T)j + T(0.5)), hiy = (T)(Ly - j) - T(0.5);
      const V2<T> u0 = interp_lin<T>(J, rho0, t0, Lx, Ly, ik, j, d[k].x, d[k].y);
      const T px = clampT(d[k].x + h * u0.x, lox, hix);
      const T py = clampT(d[k].y + h * u0.y, loy, hiy);
      const V2<T> u1 = interp_lin<T>(J, rho0, t1, Lx, Ly, ik, j, px, py);
      const T cx = clampT(d[k].x + hh * (u0.x + u1.x), lox, hix);
      const T cy = clampT(d[k].y + hh * (u0.y + u1.y), loy, hiy);
      o[k] = mk2<T>(cx, cy);
      const T ex = cx - px, ey = cy - py;
      e2 = max(e2, ex * ex + ey * ey);
      const V2<T> vn = node_v(J[p + k], rho0[p + k], t1);
      v2 = max(v2, vn.x * vn.x + vn.y * vn.y);
    }
    store_pair(dout + p, o);
  }
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  e2 = warp_max(e2);
  v2 = warp_max(v2);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&s_err2, (unsigned long long)__double_as_longlong((double)e2));
    atomicMax(&s_v2, (unsigned long long)__double_as_longlong((double)v2));
    __threadfence_block();
    const unsigned int arrived = atomicAdd(&s_warps, 1u);
    if (arrived == (blockDim.x >> 5) - 1) {
      __threadfence_block();
      atomic_max_nonneg(&st->err2_bits, __longlong_as_double((long long)atomicOr(&s_err2, 0ull)));
      atomic_max_nonneg(&st->vmax2_bits, __longlong_as_double((long long)atomicOr(&s_v2, 0ull)));
      __threadfence();
      const unsigned int tk = atomicAdd(&st->ticket, 1u);
      if (tk == gridDim.x - 1) {
        __threadfence();
        control_linear(st, sp, handle, use_cond);
      }
    }
  }
}

// max |J / rho0|^2 over the grid nodes (the speed at t = 0) into st->vmax2_bits.
template <typename T>
__global__ void linear_vmax_kernel(DevState* st, const V2<T>* J, const T* rho0, int N) {
  T v2 = T(0);
  bool bad = false;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    bad |= !(rho0[p] > T(0));
    const V2<T> v = node_v(J[p], rho0[p], T(0));
    v2 = max(v2, v.x * v.x + v.y * v.y);
  }
  v2 = warp_max(v2);
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&st->vmax2_bits, (double)v2);
    if (bad) st->bad = 1;
  }
}

// First step of a linear integration: h = min(dt0, cfl / max|v(0)|, 1).
static __global__ void linear_init_finish_kernel(DevState* st, StepParams sp, cudaGraphConditionalHandle handle,
                                                 int use_cond) {
  const double vmax = sqrt(__longlong_as_double((long long)st->vmax2_bits));
  int status = kRunning;
  double h = sp.dt0;
  if (st->bad) status = kStepFail;
  else {
    if (vmax > 0.0 && h * vmax > sp.cfl) h = sp.cfl / vmax;
    if (h > 1.0) h = 1.0;
  }
  st->vmax = vmax;
  st->h = h;
  st->status = status;
  st->err2_bits = 0;
  st->vmax2_bits = 0;
  st->dev_bits = 0;
  st->ticket = 0;
  st->bad = 0;
  if (status != kRunning && use_cond) cudaGraphSetConditional(handle, 0);
}

}  // namespace cg
