// The paper's linear-equalisation flow (SI Eq. fmn_fast: f_mn = 1 - t for t <= 1).
//
// Its flux is constant in time: with f'_mn = -1, SI Eqs. Jxmn and Jymn give
// J = -grad Phi with Phi~_mn = rho~_mn / (pi^2 (m^2/Lx^2 + n^2/Ly^2)), evaluated once per
// integration by the inverse transform passes. The density is rho(t) = (1-t) rho0 + t
// rho_bar (main text Eq. rho_ffb, rho_bar = 1 here), so the velocity at the grid points
// needs no transform per step: one elementwise kernel forms v(t1) = J / rho(t1) at every
// grid point (the paper's "basic arithmetic" at the grid points), and the same
// predictor-corrector kernel as the diffusion flow interpolates between them. The
// integration ends at t = 1.
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

// 1 / rho: in FP32 the hardware's approximate reciprocal (within 2 ulp for the positive
// normal densities here, far inside the error of the FP32 transforms that produce rho0 and
// J), in FP64 a division.
__device__ __forceinline__ float lin_recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double lin_recip(double x) { return 1.0 / x; }

// v = J / ((1 - t) rho0 + t) at every grid point, and max |v|^2 into st->vmax2_bits.
// Init mode (kModeInit): t = 0 into vbuf0 (the field at the start, parity 0), a
// non-positive rho0 flagged. Step mode (kModeLinear): the end t1 = min(t + h, 1) of the
// attempt, into the buffer that the predictor-corrector kernel reads as the new field;
// the first kernel of an attempt, so it also ends the graph loop once the integration is
// over or has run more attempts than the controller allows.
template <typename T>
__global__ void __launch_bounds__(256) linear_velocity_kernel(DevState* st, const V2<T>* __restrict__ J,
                                                               const T* __restrict__ rho0, V2<T>* vbuf0,
                                                               V2<T>* vbuf1, int N, int mode,
                                                               cudaGraphConditionalHandle handle, int use_cond,
                                                               unsigned int max_body) {
  using OB = OrdBits<T>;
  __shared__ typename OB::U s_v2;
  __shared__ unsigned int s_warps;
  __shared__ int s_run, s_par;
  __shared__ T s_t1;
  if (threadIdx.x == 0) {
    s_v2 = 0;
    s_warps = 0u;
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const bool step = mode == kModeLinear;
  if (threadIdx.x == 0) {
    // the attempt's end in the working type, converted once per block
    int run = 1, par = 0;
    double t1 = 0.0;
    if (step) {
      if (blockIdx.x == 0) {
        const unsigned int it = atomicAdd(&st->body_iters, 1u) + 1u;
        if (st->status == kRunning && it > max_body) st->status = kStepFail;
        if (st->status != kRunning && use_cond) cudaGraphSetConditional(handle, 0);
      }
      run = st->status == kRunning;
      par = st->parity;
      t1 = linear_t1(st->t, st->h);
    }
    s_run = run;
    s_par = par;
    s_t1 = (T)t1;
  }
  __syncthreads();
  if (!s_run) return;
  const T t1 = s_t1;
  V2<T>* out = step ? (s_par ? vbuf0 : vbuf1) : vbuf0;
  T v2 = T(0);
  bool bad = false;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const T r0 = rho0[p];
    bad |= !(r0 > T(0));
    const T inv = lin_recip((T(1) - t1) * r0 + t1);
    const V2<T> j = J[p];
    const V2<T> v = mk2<T>(j.x * inv, j.y * inv);
    out[p] = v;
    v2 = max(v2, v.x * v.x + v.y * v.y);
  }
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  v2 = warp_max(v2);
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (bad && !step) st->bad = 1;
    atomicMax(&s_v2, OB::of(v2));
    __threadfence_block();
    if (atomicAdd(&s_warps, 1u) == (blockDim.x >> 5) - 1) {
      __threadfence_block();
      atomic_max_nonneg(&st->vmax2_bits, OB::value(atomicOr(&s_v2, (typename OB::U)0)));
    }
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
  // set either way: inside an outer loop the same step loop runs once per iteration
  if (use_cond) cudaGraphSetConditional(handle, status == kRunning ? 1u : 0u);
}

}  // namespace cg
