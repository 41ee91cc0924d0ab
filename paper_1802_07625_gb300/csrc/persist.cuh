// One whole integration (the step loop from t = 0 to equalisation) as one cooperative
// kernel. Every block is resident; the phases of an attempted step are separated by a
// grid barrier:
//   pass 1 (spectral rows at t+h) | pass 2 (columns -> v(t+h), reductions) |
//   Heun step of all points (error reduction) | controller
// The per-attempt reductions go to one of two global slots (attempt k uses slot k&1;
// block 0 clears the other slot while deciding). Every block reads the same reduced
// values after the barrier and takes the same accept/reject decision, so the step state
// is replicated instead of broadcast. Barrier waits are bounded: a block that gives up
// records CG_ETIMEOUT's status and leaves, and the others then give up at their next
// barrier.
#pragma once

#include "advect.cuh"
#include "kernels.h"
#include "spectral.cuh"

namespace cg {

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch. `gen` is the barrier generation as seen
// by thread 0 of this block. Returns false if the wait ran out after `spins` polls.
__device__ __forceinline__ bool grid_barrier(GridBarrier* gb, unsigned int& gen, long long spins) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    // this block's global writes: visible to other blocks' loads and bulk copies
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    const unsigned int g = gen;
    const unsigned int arrived = atomicAdd(&gb->count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicExch(&gb->gen, g + 1u);
    } else {
      long long left = spins;
      while (ld_acquire_gpu(&gb->gen) == g) {
        if (--left <= 0) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    gen = g + 1u;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) {
  return atomicOr(const_cast<unsigned long long*>(p), 0ull);
}

template <typename T>
__device__ __noinline__ bool p1_dispatch(int log2N, const T* spec, V2<T>* ABt, const V2<T>* W,
                                            const V2<T>* E, int Ly, int S, int n0, double tau,
                                            unsigned char* smem, uint64_t* bar, uint32_t& ph) {
  switch (log2N) {
#define CG_P1(L) \
  case L:        \
    return p1_rows<T, L>(spec, ABt, W, E, Ly, S, n0, tau, smem, bar, ph);
    CG_P1(3) CG_P1(4) CG_P1(5) CG_P1(6) CG_P1(7) CG_P1(8) CG_P1(9) CG_P1(10)
#undef CG_P1
    default: return false;
  }
}

template <typename T>
__device__ __noinline__ bool p2_dispatch(int log2N, const V2<T>* ABt, V2<T>* out, const V2<T>* W,
                                            const V2<T>* E, int Lx, int Wc, int c0,
                                            unsigned char* smem, uint64_t* bar, uint32_t& ph,
                                            FieldRed<T>& r) {
  switch (log2N) {
#define CG_P2(L) \
  case L:        \
    return p2_cols<T, L>(ABt, out, nullptr, W, E, Lx, Wc, c0, smem, bar, ph, r);
    CG_P2(3) CG_P2(4) CG_P2(5) CG_P2(6) CG_P2(7) CG_P2(8) CG_P2(9) CG_P2(10)
#undef CG_P2
    default: return false;
  }
}

template <typename T>
__device__ __noinline__ T heun_pairs_call(const V2<T>* vcur, const V2<T>* vnew, const V2<T>* din,
                                          V2<T>* dout, int Lx, int Ly, int log2Lx, double hd, int q0,
                                          int qstride) {
  return heun_pairs<T, false>(vcur, vnew, din, dout, nullptr, nullptr, Lx, Ly, log2Lx, (T)hd, (T)(0.5 * hd), q0,
                             qstride);
}

template <typename T>
__global__ void __launch_bounds__(kIntegrateThreads) integrate_kernel(IntegrateArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ double s_h, s_tau;
  __shared__ int s_status, s_par;
  __shared__ T red[32];
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t ph = 0;
  unsigned int gen = 0;
  const int nrows = a.Ly / a.S, ncols = a.Lx / a.Wc;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthreads = gridDim.x * blockDim.x;
  const int N = a.Lx * a.Ly;

  // step state, identical in every block (kept by thread 0)
  double t = 0.0, h = a.sp.dt0, vmax = 0.0;
  long long n_acc = 0, n_rej = 0;
  int par = 0, status = kRunning, fault = 0;

  // density and velocity at tau into `out`, reductions into `slot`
  auto field = [&](double tau, V2<T>* out, StepAcc* slot) -> bool {
    for (int it = blockIdx.x; it < nrows; it += gridDim.x)
      if (!p1_dispatch<T>(a.log2Lx, a.spec, a.ABt, a.Wx, a.Ex, a.Ly, a.S, it * a.S, tau, smem, &bar, ph))
        return false;
    if (!grid_barrier(a.gb, gen, a.spins)) return false;
    T dev = T(0), v2 = T(0);
    bool bad = false;
    for (int it = blockIdx.x; it < ncols; it += gridDim.x) {
      FieldRed<T> r;
      if (!p2_dispatch<T>(a.log2Ly, a.ABt, out, a.Wy, a.Ey, a.Lx, a.Wc, it * a.Wc, smem, &bar, ph, r))
        return false;
      dev = max(dev, r.dev);
      v2 = max(v2, r.v2max);
      bad |= r.bad;
    }
    if (threadIdx.x == 0) {
      atomic_max_nonneg(&slot->dev, (double)dev);
      atomic_max_nonneg(&slot->vmax2, (double)v2);
      if (bad) atomicOr(&slot->bad, 1u);
    }
    return grid_barrier(a.gb, gen, a.spins);
  };

  // ---- field at t = 0 and the first step ----
  for (int p = tid; p < N; p += nthreads) a.d0[p] = mk2<T>(T(0), T(0));
  bool ok = field(0.0, a.v0, &a.acc[0]);
  if (ok && threadIdx.x == 0) {
    const double v2 = __longlong_as_double((long long)ld_cg_u64(&a.acc[0].vmax2));
    const double dev = __longlong_as_double((long long)ld_cg_u64(&a.acc[0].dev));
    const unsigned int bad = atomicOr(&a.acc[0].bad, 0u);
    vmax = sqrt(v2);
    if (bad) status = kStepFail;
    else if (dev <= a.sp.rho_tol) status = kDone;
    else if (vmax > 0.0 && h * vmax > a.sp.cfl) h = a.sp.cfl / vmax;
    s_status = status;
  }
  __syncthreads();
  if (ok) status = s_status;

  // ---- attempted steps ----
  long long k = 0;
  while (ok && status == kRunning) {
    ++k;
    StepAcc* slot = &a.acc[k & 1];
    if (threadIdx.x == 0) {
      s_h = h;
      s_tau = t + h;
      s_par = par;
    }
    __syncthreads();
    const double hs = s_h, tau = s_tau;
    const int ps = s_par;
    V2<T>* vcur = ps ? a.v1 : a.v0;
    V2<T>* vnew = ps ? a.v0 : a.v1;
    V2<T>* dcur = ps ? a.d1 : a.d0;
    V2<T>* dnew = ps ? a.d0 : a.d1;
    ok = field(tau, vnew, slot);
    if (!ok) break;
    T e2 = heun_pairs_call<T>(vcur, vnew, dcur, dnew, a.Lx, a.Ly, a.log2Lx, hs, tid, nthreads);
    e2 = block_max(e2, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&slot->err2, (double)e2);
    // one clock reading for all blocks: block 0 flags the slot (bit 2) before the
    // barrier, and every replicated controller reads the same flag after it
    if (blockIdx.x == 0 && threadIdx.x == 0 && deadline_passed(a.sp)) atomicOr(&slot->bad, 2u);
    ok = grid_barrier(a.gb, gen, a.spins);
    if (!ok) break;
    if (threadIdx.x == 0) {
      // the controller, replicated: accept / reject, next step, stopping rule
      const double e = sqrt(__longlong_as_double((long long)ld_cg_u64(&slot->err2)));
      const double vmax_new = sqrt(__longlong_as_double((long long)ld_cg_u64(&slot->vmax2)));
      const double dev_new = __longlong_as_double((long long)ld_cg_u64(&slot->dev));
      const unsigned int bad = atomicOr(&slot->bad, 0u);
      if (bad & 1u) {
        status = kStepFail;
      } else if (e <= a.sp.atol) {
        par ^= 1;
        t += h;
        ++n_acc;
        vmax = vmax_new;
        if (dev_new <= a.sp.rho_tol) status = kDone;
        else h *= a.sp.grow;
      } else {
        ++n_rej;
        h *= a.sp.shrink;
      }
      if (status == kRunning) {
        if (n_acc + n_rej >= a.sp.max_steps || !(h > a.sp.h_min)) status = kStepFail;
        else if (bad & 2u) status = kTimeout;
        else if (vmax > 0.0 && h * vmax > a.sp.cfl) h = a.sp.cfl / vmax;
      }
      if (blockIdx.x == 0) {
        StepAcc* other = &a.acc[(k + 1) & 1];
        atomicExch(&other->err2, 0ull);
        atomicExch(&other->vmax2, 0ull);
        atomicExch(&other->dev, 0ull);
        atomicExch(&other->bad, 0u);
      }
      s_status = status;
    }
    __syncthreads();
    status = s_status;
  }
  if (!ok) fault = 1;

  // ---- result: displacements of the current buffer, and the state ----
  if (threadIdx.x == 0) s_par = par;
  __syncthreads();
  if (!fault) {
    const V2<T>* src = s_par ? a.d1 : a.d0;
    for (int p = tid; p < N; p += nthreads) a.dres[p] = src[p];
  }
  if (threadIdx.x == 0 && (blockIdx.x == 0 || fault)) {
    if (blockIdx.x == 0) {
      a.st->t = t;
      a.st->h = h;
      a.st->vmax = vmax;
      a.st->accepted = n_acc;
      a.st->rejected = n_rej;
      a.st->parity = par;
    }
    if (fault) atomicExch(&a.st->status, kTimeout);
    else if (blockIdx.x == 0) atomicCAS(&a.st->status, kRunning, status);
  }
}

}  // namespace cg
