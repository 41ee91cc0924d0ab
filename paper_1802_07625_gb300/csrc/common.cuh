// Shared device helpers of the cartogram kernels: complex arithmetic on float2 /
// double2, order-preserving atomic max of non-negative values, block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cg {

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T> using V2 = typename vec2<T>::type;

template <typename T> __host__ __device__ __forceinline__ V2<T> mk2(T x, T y) {
  V2<T> r; r.x = x; r.y = y; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}

constexpr double kPi = 3.14159265358979323846;

// (T)i for 0 <= i < 2^22. FP32 takes the bit pattern of 1.5 * 2^23 + i and one exact add
// instead of the conversion unit; other types convert.
__device__ __forceinline__ float int_to(int i, float) {
  return __fsub_rn(__int_as_float(0x4B400000 + i), 12582912.0f);
}
template <typename A> __device__ __forceinline__ A int_to(int i, A) { return A(i); }

// Step-control constants passed by value to the kernels that need them.
struct StepParams {
  double dt0, atol, grow, shrink, cfl, rho_tol, h_min;
  long long max_steps;
  // bit pattern of the largest x >= 0 with sqrt(x) <= atol in double arithmetic (the
  // square root is correctly rounded and monotone), so that the accept test on the
  // squared error needs no FP64 square root: sqrt(e2) <= atol  <=>  bits(e2) <= this
  unsigned long long err2_accept_bits;
  double* sched;  // if not null: (t, h) of every accepted step, [max_steps][2]
  // if not null: device-clock deadline of the call in ns (0: none), written at its start
  const unsigned long long* deadline;
};

// Step state of the diffusion flow's step loop (graph and host-driven modes), kept in
// two slots by attempt parity: slot b holds the state at the start of an attempt of
// parity b and that attempt's reductions. Every block of the first pass of attempt n
// computes the controller's decision on attempt n - 1 from slot (n - 1) & 1 (so the
// decision needs no serial tail at the end of the step kernel); its block 0 stores the
// result into slot n & 1, which pass 2 and the step kernel of attempt n read. One slot
// per 128-byte line.
struct __align__(128) LoopSlot {
  double t, h, vmax;
  long long accepted, rejected;
  int parity, status;
  int pending;  // an attempt ran from this state: its reductions are below
  int bad;      // bit 0: the new field's density was not positive; bit 1: deadline passed
  unsigned long long err2_bits;   // max ||r_corr - r_pred||^2
  unsigned long long vmax2_bits;  // max |v|^2 of the new field
  unsigned long long dev_bits;    // max |rho/rho_bar - 1| of the new field
};

// Device-resident state of one integration (written by the step controller).
struct DevState {
  double t;          // accepted diffusion time
  double h;          // step to attempt next (already capped)
  double vmax;       // max |v| of the field at t
  long long accepted;
  long long rejected;
  int parity;        // current buffers: v[parity], disp[parity]
  int status;        // kRunning, kDone, or a negative error code
  // reductions of the attempt in flight (bit patterns of non-negative doubles)
  unsigned long long err2_bits;   // max ||r_corr - r_pred||^2
  unsigned long long vmax2_bits;  // max |v|^2 of the new field
  unsigned long long dev_bits;    // max |rho/rho_bar - 1| of the new field
  unsigned int ticket;            // blocks of the step kernel that have finished
  int bad;                        // a field had a non-positive or non-finite density
  unsigned int body_iters;        // step-loop iterations started (termination guard)
  unsigned int pad;
  unsigned long long t_start_ns;  // device clock at the start of the integration
  StepParams sp;                  // the integration's constants (written at its start)
  LoopSlot ls[2];                 // the step loop's state by attempt parity
};
// What a field or step kernel works on: the field at t (start of an integration),
// the attempt at t + h inside the step loop, or explicit buffers and times.
enum FieldMode { kModeInit = 0, kModeStep = 1, kModeFixed = 2, kModeFlux = 3, kModeLinear = 4, kModeStepOdd = 5 };
// kModeStep / kModeStepOdd: an attempt of the diffusion flow's step loop of even / odd
// parity (its state in DevState::ls).
__host__ __device__ inline bool is_step_mode(int mode) { return mode == kModeStep || mode == kModeStepOdd; }
__host__ __device__ inline int step_slot(int mode) { return mode == kModeStepOdd ? 1 : 0; }
// kModeFlux: explicit buffers like kModeFixed, and pass 2 writes -grad instead of the
// velocity (the flux J = -grad Phi of the linear-equalisation flow).
// kModeLinear: a step-loop attempt of the linear-equalisation flow (buffers by parity,
// the attempt ends at min(t + h, 1), its own controller).

constexpr int kRunning = 0;
constexpr int kDone = 1;
constexpr int kStepFail = -6;
constexpr int kTimeout = -7;

// Per-iteration results read back by the host in one copy.
// Fixed-size chunks of the rings' vertices for the shoelace area sums (built with the
// map): chunk c covers up to kAreaChunk consecutive vertices of ring chunk_ring[c]; ring
// k's chunks are [ring_chunk_off[k], ring_chunk_off[k+1]); chunk_sum holds one partial
// sum per chunk.
constexpr int kAreaChunk = 64;
struct AreaChunks {
  const int* chunk_ring;
  const int* ring_chunk_off;
  long long n_chunks;
  double* chunk_sum;
};

struct IterInfo {
  double max_err;       // max_i |A_i / A^_i - 1|
  double t_end;         // diffusion time reached by the integration
  long long accepted;
  long long rejected;
  int status;           // DevState status after the integration
  int pad;
  unsigned long long loop_ns;  // device time of the integration (init to finish)
};

// What an outer iteration leaves behind with its projected grid (stored after the grid in
// the iteration's history slot): the largest relative area error once the vertices are
// mapped, the integration's end time and step counts, its device time and blur width.
struct IterRecord {
  double max_err;
  double t_end;
  double blur;
  long long accepted;
  long long rejected;
  unsigned long long loop_ns;
};

// State of the outer iteration when it runs on the device (one CUDA-graph launch runs
// iterations until the areas converge, the budget ends, an integration fails, or the
// history has no free slot). Written by the host before a launch, read after it.
struct OuterState {
  void** hist;                // device pointers of the projected-grid history slots
  const double* sigma;        // blur width of each iteration of this call
  double area_tol;
  double max_err;             // max |A_i / A^_i - 1| of the current map
  double t_end;               // end time of the last integration
  long long accepted;         // attempted steps of this call's integrations
  long long rejected;
  unsigned long long loop_ns; // device time of this call's integrations
  int k;                      // history length = slot of the next projected grid
  int cap;                    // slots allocated
  int iterations;             // iterations of this call
  int max_iter;               // iteration budget of this call
  int status;                 // kOuter* below, or a failed integration's status (< 0)
  int pad;
  unsigned long long rec_offset;  // byte offset of the IterRecord in a history slot
};
constexpr int kOuterRunning = 0;
constexpr int kOuterConverged = 1;
constexpr int kOuterNeedSlots = 2;
constexpr int kOuterNoConverge = -4;

// Device clock in nanoseconds.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier state of the persistent integration kernel.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

struct StepAcc {
  unsigned long long err2;   // max ||r_corr - r_pred||^2 (bits of a non-negative double)
  unsigned long long vmax2;  // max |v|^2 of the new field
  unsigned long long dev;    // max |rho/rho_bar - 1| of the new field
  unsigned int bad;          // a non-positive or non-finite density
  unsigned int pad;
};


// The call's deadline has passed (read by the step controllers after every attempt).
__device__ __forceinline__ bool deadline_passed(const StepParams& sp) {
  if (!sp.deadline) return false;
  const unsigned long long d = *(volatile const unsigned long long*)sp.deadline;
  return d != 0ull && global_ns() > d;
}

// A loop slot as written by other blocks or earlier kernels: every field from L2.
__device__ __forceinline__ LoopSlot load_slot(const LoopSlot* q) {
  LoopSlot r;
  r.t = __ldcg(&q->t);
  r.h = __ldcg(&q->h);
  r.vmax = __ldcg(&q->vmax);
  r.accepted = __ldcg(&q->accepted);
  r.rejected = __ldcg(&q->rejected);
  r.parity = __ldcg(&q->parity);
  r.status = __ldcg(&q->status);
  r.pending = __ldcg(&q->pending);
  r.bad = __ldcg(&q->bad);
  r.err2_bits = __ldcg(&q->err2_bits);
  r.vmax2_bits = __ldcg(&q->vmax2_bits);
  r.dev_bits = __ldcg(&q->dev_bits);
  return r;
}

// The integration's constants as stored in its state, from L2.
__device__ __forceinline__ StepParams load_sp(const DevState* st) {
  StepParams r;
  r.dt0 = __ldcg(&st->sp.dt0);
  r.atol = __ldcg(&st->sp.atol);
  r.grow = __ldcg(&st->sp.grow);
  r.shrink = __ldcg(&st->sp.shrink);
  r.cfl = __ldcg(&st->sp.cfl);
  r.rho_tol = __ldcg(&st->sp.rho_tol);
  r.h_min = __ldcg(&st->sp.h_min);
  r.max_steps = __ldcg(&st->sp.max_steps);
  r.err2_accept_bits = __ldcg(&st->sp.err2_accept_bits);
  r.sched = (double*)__ldcg((const long long*)&st->sp.sched);
  r.deadline = (const unsigned long long*)__ldcg((const long long*)&st->sp.deadline);
  return r;
}

// The step controller (the paper's predictor-corrector "automatically adapts the size
// of the next time step") on the attempt run from state p, whose reductions p holds:
// accept if max ||r_corr - r_pred|| <= atol (t += h; the integration ends once
// max |rho/rho_bar - 1| <= rho_tol, else h *= grow), otherwise h *= shrink; the step
// budget or a collapsed step end it with a failure, a passed deadline with a time-out;
// the next step is capped by h * max|v| <= cfl with the field at the accepted time.
// Returns the state at the start of the next attempt (reductions cleared). Pure: every
// kernel of that attempt computes it from the same slot and gets the same answer.
// `record`: store each accepted (t, h) into sp.sched (one caller only).
__device__ __forceinline__ LoopSlot loop_decide(const LoopSlot& p, const StepParams& sp, bool record) {
  LoopSlot n = p;
  n.bad = 0;
  n.err2_bits = 0;
  n.vmax2_bits = 0;
  n.dev_bits = 0;
  n.pending = 0;
  if (p.status != kRunning) return n;
  n.pending = 1;
  if (!p.pending) return n;  // the integration's first attempt
  // The decision is on the critical path of every attempt and GB300's FP64 pipe is
  // narrow: the accept and stop tests compare bit patterns of non-negative doubles
  // (ordered like their values), and the new field's speed (a square root) is taken
  // only on acceptance. The outcome is that of the plain formulas: accept iff
  // sqrt(err2) <= atol; done iff dev <= rho_tol; cap h at cfl / vmax.
  int status = kRunning;
  double h = p.h;
  if (p.bad & 1) {
    status = kStepFail;
  } else if (p.err2_bits <= sp.err2_accept_bits) {
    if (record && sp.sched) {
      sp.sched[2 * p.accepted] = p.t;
      sp.sched[2 * p.accepted + 1] = h;
    }
    n.parity = p.parity ^ 1;
    n.t = p.t + h;
    n.accepted = p.accepted + 1;
    n.vmax = sqrt(__longlong_as_double((long long)p.vmax2_bits));
    if (p.dev_bits <= (unsigned long long)__double_as_longlong(sp.rho_tol)) status = kDone;
    else h *= sp.grow;
  } else {
    n.rejected = p.rejected + 1;
    h *= sp.shrink;
  }
  if (status == kRunning) {
    if (n.accepted + n.rejected >= sp.max_steps || !(h > sp.h_min)) status = kStepFail;
    else if (p.bad & 2) status = kTimeout;
    else if (n.vmax > 0.0 && h * n.vmax > sp.cfl) h = sp.cfl / n.vmax;
  }
  n.h = h;
  n.status = status;
  if (status != kRunning) n.pending = 0;
  return n;
}

// Bit patterns of non-negative values in the working type's own width (they order like
// the values), so that block reductions convert to FP64 once per block, not per warp:
// GB300's FP64 pipe is narrow, and every conversion to or from double uses it.
template <typename T> struct OrdBits;
template <> struct OrdBits<float> {
  using U = unsigned int;
  static __device__ __forceinline__ U of(float v) { return __float_as_uint(v); }
  static __device__ __forceinline__ double value(U u) { return (double)__uint_as_float(u); }
};
template <> struct OrdBits<double> {
  using U = unsigned long long;
  static __device__ __forceinline__ U of(double v) { return (U)__double_as_longlong(v); }
  static __device__ __forceinline__ double value(U u) { return __longlong_as_double((long long)u); }
};

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Max over the block; the result is valid in thread 0. `red` holds >= 32 values.
template <typename T> __device__ __forceinline__ T block_max(T v, T* red) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? red[lane] : T(0);
    v = warp_max(v);
  }
  return v;
}

// Arguments of the persistent integration kernel.
template <typename T>
struct IntegrateArgs {
  const T* spec;
  V2<T>* ABt;
  const V2<T>* Wx;
  const V2<T>* Ex;
  const V2<T>* Wy;
  const V2<T>* Ey;
  V2<T>* v0;
  V2<T>* v1;
  V2<T>* d0;
  V2<T>* d1;
  V2<T>* dres;
  DevState* st;
  GridBarrier* gb;
  StepAcc* acc;  // two slots, zero at launch
  StepParams sp;
  int Lx, Ly, log2Lx, log2Ly, S, Wc;
  long long spins;  // polls of one grid-barrier wait before giving up
};

}  // namespace cg
