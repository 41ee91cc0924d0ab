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

// floor(x), as an integer and as a value of x's type. For FP32 it takes full-rate adds
// instead of the conversion unit: x + 1.5 * 2^23 rounded toward -inf holds floor(x) in
// its low mantissa bits, exactly for |x| < 2^22 (every displacement here is below the
// grid size). Other values (huge, infinite, NaN) give some integer, in unsigned
// arithmetic, which the callers' range tests and index clamps keep inside the grid.
__device__ __forceinline__ unsigned floor_parts(float x, float& fl) {
  const float t = __fadd_rd(x, 12582912.0f);
  fl = __fsub_rn(t, 12582912.0f);
  return (unsigned)__float_as_int(t) - 0x4B400000u;
}
__device__ __forceinline__ unsigned floor_parts(double x, double& fl) {
  fl = min(max(floor(x), -4194304.0), 4194304.0);
  return (unsigned)(int)fl;
}
// Cell of the interpolation lattice that holds the grid point (i, j) displaced by
// (dx, dy): lower-left grid point (ix, iy) and the fractions (fx, fy).
template <typename T> struct Cell {
  int ix, iy;
  T fx, fy;
};
template <typename T>
__device__ __forceinline__ Cell<T> cell_of(int i, int j, T dx, T dy) {
  T flx, fly;
  Cell<T> c;
  c.ix = (int)((unsigned)i + floor_parts(dx, flx));
  c.iy = (int)((unsigned)j + floor_parts(dy, fly));
  c.fx = dx - flx;
  c.fy = dy - fly;
  return c;
}
template <typename T> __device__ __forceinline__ bool cell_inside(const Cell<T>& c, int Lx, int Ly) {
  return (unsigned)c.ix < (unsigned)(Lx - 1) && (unsigned)c.iy < (unsigned)(Ly - 1);
}

// The velocities at the four corners of a cell: (ix, iy), (ix+1, iy), (ix, iy+1),
// (ix+1, iy+1), with the indices clamped to the grid next to a wall (the tangential
// velocity of the nearest grid point).
template <typename T> struct Quad {
  V2<T> a, b, c, d;
};
template <typename T>
__device__ __forceinline__ Quad<T> load_quad(const V2<T>* __restrict__ v, int Lx, int Ly, const Cell<T>& c) {
  Quad<T> q;
  if (cell_inside(c, Lx, Ly)) {
    // a cell between four grid points (almost every point): no clamping
    const V2<T>* r0 = v + (c.iy * Lx + c.ix);  // Lx * Ly < 2^31
    const V2<T>* r1 = r0 + Lx;
    q.a = __ldg(r0);
    q.b = __ldg(r0 + 1);
    q.c = __ldg(r1);
    q.d = __ldg(r1 + 1);
    return q;
  }
  const int i0 = min(max(c.ix, 0), Lx - 1), i1 = min(max(c.ix + 1, 0), Lx - 1);
  const int j0 = min(max(c.iy, 0), Ly - 1), j1 = min(max(c.iy + 1, 0), Ly - 1);
  const int r0 = j0 * Lx, r1 = j1 * Lx;
  q.a = __ldg(v + r0 + i0);
  q.b = __ldg(v + r0 + i1);
  q.c = __ldg(v + r1 + i0);
  q.d = __ldg(v + r1 + i1);
  return q;
}

// Bilinear combination of a cell's corner velocities at the fractions of `c`, with
// explicit fused multiply-adds (every caller rounds the same way). Next to a wall the
// normal component is scaled down to zero at the wall: v_x by min(1, 2x, 2(Lx - x)),
// v_y likewise, where (x, y) = (i + 1/2 + dx, j + 1/2 + dy).
template <typename T>
__device__ __forceinline__ V2<T> bilerp(const Quad<T>& q, const Cell<T>& c, int i, int j, T dx, T dy, int Lx,
                                        int Ly) {
  const T gx = T(1) - c.fx, gy = T(1) - c.fy;
  const T lox = fma(gx, q.a.x, c.fx * q.b.x), hix = fma(gx, q.c.x, c.fx * q.d.x);
  const T loy = fma(gx, q.a.y, c.fx * q.b.y), hiy = fma(gx, q.c.y, c.fx * q.d.y);
  T ux = fma(gy, lox, c.fy * hix);
  T uy = fma(gy, loy, c.fy * hiy);
  if (!cell_inside(c, Lx, Ly)) {
    const T x = (T)i + T(0.5) + dx, y = (T)j + T(0.5) + dy;
    if (c.ix < 0 || c.ix >= Lx - 1) ux *= min(T(1), min(T(2) * x, T(2) * ((T)Lx - x)));
    if (c.iy < 0 || c.iy >= Ly - 1) uy *= min(T(1), min(T(2) * y, T(2) * ((T)Ly - y)));
  }
  return mk2<T>(ux, uy);
}

// Velocity field v interpolated at grid point (i, j) displaced by (dx, dy).
template <typename T>
__device__ __forceinline__ V2<T> interp_v(const V2<T>* __restrict__ v, int Lx, int Ly, int i, int j,
                                         T dx, T dy) {
  const Cell<T> c = cell_of<T>(i, j, dx, dy);
  return bilerp<T>(load_quad<T>(v, Lx, Ly, c), c, i, j, dx, dy, Lx, Ly);
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
// CACHED: the predictor's velocity v(t) at each point's position is read from uin
// instead of being interpolated, and v(t + h) at the corrected position is written to
// uout for the next attempt (a point's own value, so its loads and stores are
// coalesced). The corrected position lies within the step error of the predicted one,
// so it almost always falls in the same cell, whose four corner velocities the
// corrector has just gathered: only the bilinear weights change. A rejected attempt
// leaves uin as it was, and the retry from the same positions reads it again. This
// removes one of the three dependent rounds of loads per point; the values are the
// ones interpolation would give (same corners, same arithmetic).
// h and hh = h/2 are the step in the working type, as (T)h and (T)(0.5 h) of the FP64 step.
template <typename T, bool CACHED>
__device__ __forceinline__ T heun_pairs(const V2<T>* __restrict__ vcur, const V2<T>* __restrict__ vnew,
                                        const V2<T>* __restrict__ din, V2<T>* __restrict__ dout,
                                        const V2<T>* __restrict__ uin, V2<T>* __restrict__ uout, int Lx,
                                        int Ly, int log2Lx, T h, T hh, int q0, int qstride) {
  const int npairs = (Lx * Ly) >> 1;
  const T Lxh = (T)Lx - T(0.5), Lyh = (T)Ly - T(0.5);
  T e2 = T(0);
  // two horizontally adjacent points per thread (Lx is even), one vector load/store
  for (int q = q0; q < npairs; q += qstride) {
    const int p = 2 * q;
    const int i = p & (Lx - 1), j = p >> log2Lx;
    V2<T> d[2], u0[2];
    load_pair(din + p, d);
    if constexpr (CACHED) load_pair(uin + p, u0);
    V2<T> o[2], un[2];
    // displacement bounds that keep a point inside the box [0, Lx] x [0, Ly]
    const T fi = int_to(i, T(0)), fj = int_to(j, T(0));
    const T loy = -(fj + T(0.5)), hiy = Lyh - fj;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int ik = i + k;
      const T lox = -(fi + (T(k) + T(0.5))), hix = (Lxh - fi) - T(k);
      if constexpr (!CACHED) u0[k] = interp_v<T>(vcur, Lx, Ly, ik, j, d[k].x, d[k].y);
      const T px = clampT(d[k].x + h * u0[k].x, lox, hix);
      const T py = clampT(d[k].y + h * u0[k].y, loy, hiy);
      const Cell<T> cp = cell_of<T>(ik, j, px, py);
      const Quad<T> qp = load_quad<T>(vnew, Lx, Ly, cp);
      const V2<T> u1 = bilerp<T>(qp, cp, ik, j, px, py, Lx, Ly);
      const T cx = clampT(d[k].x + hh * (u0[k].x + u1.x), lox, hix);
      const T cy = clampT(d[k].y + hh * (u0[k].y + u1.y), loy, hiy);
      o[k] = mk2<T>(cx, cy);
      const T ex = cx - px, ey = cy - py;
      e2 = max(e2, ex * ex + ey * ey);
      if constexpr (CACHED) {
        const Cell<T> cc = cell_of<T>(ik, j, cx, cy);
        if (cc.ix == cp.ix && cc.iy == cp.iy) un[k] = bilerp<T>(qp, cc, ik, j, cx, cy, Lx, Ly);
        else un[k] = bilerp<T>(load_quad<T>(vnew, Lx, Ly, cc), cc, ik, j, cx, cy, Lx, Ly);
      }
    }
    store_pair(dout + p, o);
    if constexpr (CACHED) store_pair(uout + p, un);
  }
  return e2;
}

// v interpolated at every displaced grid point: the cached predictor velocities of the
// first attempt of an integration.
template <typename T>
__global__ void __launch_bounds__(256) gather_u_kernel(const V2<T>* __restrict__ v, const V2<T>* __restrict__ d,
                                                       V2<T>* __restrict__ u, int Lx, int Ly, int log2Lx) {
  const int N = Lx * Ly;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const V2<T> dp = d[p];
    u[p] = interp_v<T>(v, Lx, Ly, p & (Lx - 1), p >> log2Lx, dp.x, dp.y);
  }
}

// One Heun step of every grid point. Diffusion-flow step modes (kModeStep,
// kModeStepOdd): buffers by parity and h from the attempt's state, which its first pass
// decided and stored; the step error goes to the attempt's slot, on which the next
// attempt's first pass decides.
// kModeLinear (linear-equalisation flow, the attempt ending at min(t + h, 1)): buffers
// and h from the state, and the last block to finish runs the controller. Fixed mode
// (single step on explicit buffers): vcur = vbuf0, vnew = vbuf1, din = dbuf0,
// dout = dbuf1, step h. CACHED: the predictor velocities come from ubuf (selected by
// parity like dbuf: ubuf[p] holds v(t) at the positions in dbuf[p]), and the next
// ones are written to the other ubuf; otherwise they are interpolated and ubuf is
// not touched.
template <typename T, bool CACHED>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 1) heun_kernel(DevState* st, StepParams sp,
                                                    const V2<T>* vbuf0, const V2<T>* vbuf1,
                                                    V2<T>* dbuf0, V2<T>* dbuf1, V2<T>* ubuf0,
                                                    V2<T>* ubuf1, int Lx, int Ly, int log2Lx, int mode,
                                                    double h_fixed, cudaGraphConditionalHandle handle,
                                                    int use_cond) {
  using OB = OrdBits<T>;
  __shared__ typename OB::U s_err2;
  __shared__ unsigned int s_warps;
  __shared__ int s_run, s_par;
  __shared__ T s_h[2];
  const bool pipe = is_step_mode(mode);
  const bool step = mode == kModeLinear;
  if (threadIdx.x == 0) {
    s_err2 = 0;
    s_warps = 0u;
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the fields of the previous kernel
  if (threadIdx.x == 0) {
    // the attempt's state, as its first pass decided and stored it; the step in the
    // working type is converted once per block (not per thread: FP64 is slow here)
    double hd = h_fixed;
    int run = 1, par = 0;
    if (pipe) {
      const LoopSlot* q = &st->ls[step_slot(mode)];
      run = __ldcg(&q->status) == kRunning;
      par = __ldcg(&q->parity);
      hd = __ldcg(&q->h);
    } else if (step) {
      run = st->status == kRunning;
      par = st->parity;
      hd = linear_t1(st->t, st->h) - st->t;
    }
    s_run = run;
    s_par = par;
    s_h[0] = (T)hd;
    s_h[1] = (T)(0.5 * hd);
  }
  __syncthreads();
  if (!s_run) return;
  const V2<T>* vcur = vbuf0;
  const V2<T>* vnew = vbuf1;
  const V2<T>* din = dbuf0;
  V2<T>* dout = dbuf1;
  const V2<T>* uin = ubuf0;
  V2<T>* uout = ubuf1;
  if (step || pipe) {
    const int par = s_par;
    vcur = par ? vbuf1 : vbuf0;
    vnew = par ? vbuf0 : vbuf1;
    din = par ? dbuf1 : dbuf0;
    dout = par ? dbuf0 : dbuf1;
    uin = par ? ubuf1 : ubuf0;
    uout = par ? ubuf0 : ubuf1;
  }
  T e2 = heun_pairs<T, CACHED>(vcur, vnew, din, dout, uin, uout, Lx, Ly, log2Lx, s_h[0], s_h[1],
                               blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // Block reduction without a block-wide barrier: each warp folds its maximum into
  // shared memory; the last warp of the block to arrive publishes the block maximum
  // (in the linear flow it also takes the block's ticket, and the last block runs the
  // controller).
  e2 = warp_max(e2);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&s_err2, OB::of(e2));
    __threadfence_block();
    const unsigned int arrived = atomicAdd(&s_warps, 1u);
    if (arrived == (blockDim.x >> 5) - 1) {
      __threadfence_block();
      const double bm = OB::value(atomicOr(&s_err2, (typename OB::U)0));
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
