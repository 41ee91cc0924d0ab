// Advection of all Lx*Ly grid points by one predictor-corrector step (main text Eq.
// rt_diff, integrated "using a predictor-corrector method that automatically adapts
// the size of the next time step", with "interpolating between the grid points"),
// and the device-side step controller.
//
// Positions are stored as displacements from the cell centres (i + 1/2, j + 1/2), so
// in FP32 their rounding is relative to the displacement, not to the coordinate.
// Interpolation lattice: the cell centres plus the walls x = 0, Lx and y = 0, Ly,
// where the normal velocity vanishes (no flux through the box edges) and the
// tangential velocity equals that of the nearest grid point. This is bilinear
// interpolation with indices clamped to the grid, followed by a factor
// min(1, 2x, 2(Lx - x)) on v_x (and likewise on v_y) inside the half-cell band.
#pragma once

#include "common.cuh"

namespace cg {

template <typename T>
__device__ __forceinline__ V2<T> interp_v(const V2<T>* __restrict__ v, int Lx, int Ly, int i, int j,
                                         T dx, T dy) {
  // cell of the interpolation lattice; floors are clamped before the integer
  // conversion and the indices clamped to the grid, so every load stays in bounds
  const T flx = min(max(floor(dx), T(-2 - Lx)), T(Lx + 2));
  const T fly = min(max(floor(dy), T(-2 - Ly)), T(Ly + 2));
  const int ix = i + (int)flx, iy = j + (int)fly;
  const T fx = dx - flx, fy = dy - fly;
  const T gx = T(1) - fx, gy = T(1) - fy;
  if (ix >= 0 && ix < Lx - 1 && iy >= 0 && iy < Ly - 1) {
    // a cell between four grid points (almost every point): no clamping, no wall factor
    const V2<T>* r0 = v + (iy * Lx + ix);  // Lx * Ly < 2^31
    const V2<T>* r1 = r0 + Lx;
    const V2<T> a = __ldg(r0), b = __ldg(r0 + 1);
    const V2<T> c = __ldg(r1), d = __ldg(r1 + 1);
    return mk2<T>(gy * (gx * a.x + fx * b.x) + fy * (gx * c.x + fx * d.x),
                  gy * (gx * a.y + fx * b.y) + fy * (gx * c.y + fx * d.y));
  }
  // next to a wall: the indices clamped to the grid (the tangential velocity of the
  // nearest grid point), the normal component scaled down to zero at the wall
  const int i0 = min(max(ix, 0), Lx - 1), i1 = min(max(ix + 1, 0), Lx - 1);
  const int j0 = min(max(iy, 0), Ly - 1), j1 = min(max(iy + 1, 0), Ly - 1);
  const int r0 = j0 * Lx, r1 = j1 * Lx;
  const V2<T> a = __ldg(v + r0 + i0), b = __ldg(v + r0 + i1);
  const V2<T> c = __ldg(v + r1 + i0), d = __ldg(v + r1 + i1);
  T ux = gy * (gx * a.x + fx * b.x) + fy * (gx * c.x + fx * d.x);
  T uy = gy * (gx * a.y + fx * b.y) + fy * (gx * c.y + fx * d.y);
  const T x = (T)i + T(0.5) + dx, y = (T)j + T(0.5) + dy;
  if (ix < 0 || ix >= Lx - 1) ux *= min(T(1), min(T(2) * x, T(2) * ((T)Lx - x)));
  if (iy < 0 || iy >= Ly - 1) uy *= min(T(1), min(T(2) * y, T(2) * ((T)Ly - y)));
  return mk2<T>(ux, uy);
}

// Two consecutive 2-vectors with one 16-byte access (FP32) or two (FP64).
__device__ __forceinline__ void load_pair(const float2* p, float2 (&d)[2]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  d[0] = make_float2(v.x, v.y);
  d[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void load_pair(const double2* p, double2 (&d)[2]) {
  d[0] = p[0];
  d[1] = p[1];
}
__device__ __forceinline__ void store_pair(float2* p, const float2 (&d)[2]) {
  *reinterpret_cast<float4*>(p) = make_float4(d[0].x, d[0].y, d[1].x, d[1].y);
}
__device__ __forceinline__ void store_pair(double2* p, const double2 (&d)[2]) {
  p[0] = d[0];
  p[1] = d[1];
}

template <typename T> __device__ __forceinline__ T clampT(T v, T lo, T hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// End of the attempted step t -> t1 of the linear-equalisation flow (the step that
// reaches t = 1 ends exactly there).
__device__ __forceinline__ double linear_t1(double t, double h) { return (t + h >= 1.0) ? 1.0 : t + h; }

// Controller of the linear-equalisation flow: accept / reject as for the diffusion flow
// (loop_decide), the next step capped by cfl / max|v| and by 1 - t; done once an
// accepted step reaches t = 1.
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
    else if (deadline_passed(sp)) status = kTimeout;
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

// Heun step of the point pairs q = q0, q0 + qstride, ... (two horizontally adjacent
// points per pair, Lx even); returns this thread's max ||r_corr - r_pred||^2.
template <typename T>
__device__ __forceinline__ T heun_pairs(const V2<T>* __restrict__ vcur, const V2<T>* __restrict__ vnew,
                                        const V2<T>* __restrict__ din, V2<T>* __restrict__ dout, int Lx,
                                        int Ly, int log2Lx, double hd, int q0, int qstride) {
  const T h = (T)hd, hh = (T)(0.5 * hd);
  const int npairs = (Lx * Ly) >> 1;
  T e2 = T(0);
  // two horizontally adjacent points per thread (Lx is even), one vector load/store
  for (int q = q0; q < npairs; q += qstride) {
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
      const V2<T> u0 = interp_v<T>(vcur, Lx, Ly, ik, j, d[k].x, d[k].y);
      const T px = clampT(d[k].x + h * u0.x, lox, hix);
      const T py = clampT(d[k].y + h * u0.y, loy, hiy);
      const V2<T> u1 = interp_v<T>(vnew, Lx, Ly, ik, j, px, py);
      const T cx = clampT(d[k].x + hh * (u0.x + u1.x), lox, hix);
      const T cy = clampT(d[k].y + hh * (u0.y + u1.y), loy, hiy);
      o[k] = mk2<T>(cx, cy);
      const T ex = cx - px, ey = cy - py;
      e2 = max(e2, ex * ex + ey * ey);
    }
    store_pair(dout + p, o);
  }
  return e2;
}

// One Heun step of every grid point. Diffusion-flow step modes (kModeStep,
// kModeStepOdd): buffers by parity and h from the attempt's state, which its first pass
// decided and stored; the step error goes to the attempt's slot, on which the next
// attempt's first pass decides.
// kModeLinear (linear-equalisation flow, the attempt ending at min(t + h, 1)): buffers
// and h from the state, and the last block to finish runs the controller. Fixed mode
// (single step on explicit buffers): vcur = vbuf0, vnew = vbuf1, din = dbuf0,
// dout = dbuf1, step h.
template <typename T>
__global__ void __launch_bounds__(256) heun_kernel(DevState* st, StepParams sp,
                                                    const V2<T>* vbuf0, const V2<T>* vbuf1,
                                                    V2<T>* dbuf0, V2<T>* dbuf1, int Lx, int Ly,
                                                    int log2Lx, int mode, double h_fixed,
                                                    cudaGraphConditionalHandle handle, int use_cond) {
  __shared__ unsigned long long s_err2;
  __shared__ unsigned int s_warps;
  __shared__ int s_run, s_par;
  __shared__ double s_h;
  const bool pipe = is_step_mode(mode);
  if (threadIdx.x == 0) {
    s_err2 = 0ull;
    s_warps = 0u;
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the fields of the previous kernel
  if (pipe && threadIdx.x == 0) {
    // the attempt's state, as its first pass decided and stored it
    const LoopSlot* q = &st->ls[step_slot(mode)];
    s_run = __ldcg(&q->status) == kRunning;
    s_par = __ldcg(&q->parity);
    s_h = __ldcg(&q->h);
  }
  __syncthreads();
  const bool step = mode == kModeLinear;
  if (step && st->status != kRunning) return;
  if (pipe && !s_run) return;
  const V2<T>* vcur = vbuf0;
  const V2<T>* vnew = vbuf1;
  const V2<T>* din = dbuf0;
  V2<T>* dout = dbuf1;
  double hd = h_fixed;
  if (step || pipe) {
    const int par = pipe ? s_par : st->parity;
    vcur = par ? vbuf1 : vbuf0;
    vnew = par ? vbuf0 : vbuf1;
    din = par ? dbuf1 : dbuf0;
    dout = par ? dbuf0 : dbuf1;
    hd = pipe ? s_h : linear_t1(st->t, st->h) - st->t;
  }
  T e2 = heun_pairs<T>(vcur, vnew, din, dout, Lx, Ly, log2Lx, hd,
                       blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // Block reduction without a block-wide barrier: each warp folds its maximum into
  // shared memory; the last warp of the block to arrive publishes the block maximum
  // (in the linear flow it also takes the block's ticket, and the last block runs the
  // controller).
  e2 = warp_max(e2);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&s_err2, (unsigned long long)__double_as_longlong((double)e2));
    __threadfence_block();
    const unsigned int arrived = atomicAdd(&s_warps, 1u);
    if (arrived == (blockDim.x >> 5) - 1) {
      __threadfence_block();
      const double bm = __longlong_as_double((long long)atomicOr(&s_err2, 0ull));
      if (pipe) {
        LoopSlot* q = &st->ls[step_slot(mode)];
        atomic_max_nonneg(&q->err2_bits, bm);
        // one clock reading per attempt, taken into the slot so that every kernel of
        // the next attempt decides the same
        if (blockIdx.x == 0 && deadline_passed(sp)) atomicOr(&q->bad, 2);
        return;
      }
      atomic_max_nonneg(&st->err2_bits, bm);
      if (step) {
        __threadfence();
        const unsigned int t = atomicAdd(&st->ticket, 1u);
        if (t == gridDim.x - 1) {
          __threadfence();
          control_linear(st, sp, handle, use_cond);
        }
      }
    }
  }
}

// Reset the state for a new integration (t = 0, h = dt0, parity 0, counters 0).
static __global__ void init_state_kernel(DevState* st, StepParams sp) {
  st->t = 0.0;
  st->h = sp.dt0;
  st->vmax = 0.0;
  st->accepted = 0;
  st->rejected = 0;
  st->parity = 0;
  st->status = kRunning;
  st->err2_bits = 0;
  st->vmax2_bits = 0;
  st->dev_bits = 0;
  st->ticket = 0;
  st->bad = 0;
  st->body_iters = 0;
  st->t_start_ns = global_ns();
  st->sp = sp;
}

// After the field at t = 0: stop at once if the density is already equal, else cap
// the first step.
static __global__ void init_finish_kernel(DevState* st, StepParams sp, cudaGraphConditionalHandle handle,
                                   int use_cond) {
  const double vmax = sqrt(__longlong_as_double((long long)st->vmax2_bits));
  const double dev = __longlong_as_double((long long)st->dev_bits);
  int status = kRunning;
  double h = sp.dt0;
  if (st->bad) status = kStepFail;
  else if (dev <= sp.rho_tol) status = kDone;
  else if (vmax > 0.0 && h * vmax > sp.cfl) h = sp.cfl / vmax;
  st->vmax = vmax;
  st->h = h;
  st->status = status;
  st->err2_bits = 0;
  st->vmax2_bits = 0;
  st->dev_bits = 0;
  st->ticket = 0;
  st->bad = 0;
  // the diffusion flow's step loop starts from slot 1 (the first attempt has parity 0)
  LoopSlot z = {};
  z.t = st->t;
  z.vmax = vmax;
  z.h = h;
  z.parity = st->parity;
  z.status = status;
  st->ls[1] = z;
  st->ls[0] = LoopSlot{};
  // set either way: inside an outer loop the same step loop runs once per iteration
  if (use_cond) cudaGraphSetConditional(handle, status == kRunning ? 1u : 0u);
}

// Copy the displacements of the current buffer (selected by parity) to `dst`.
template <typename T>
__global__ void snapshot_kernel(const DevState* st, const V2<T>* dbuf0, const V2<T>* dbuf1,
                                V2<T>* dst, int N) {
  const V2<T>* src = st->parity ? dbuf1 : dbuf0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) dst[p] = src[p];
}

}  // namespace cg
