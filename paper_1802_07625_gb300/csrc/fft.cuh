// Shared-memory batched complex FFT for power-of-two lengths 8..1024.
//
// A length-N transform is split four-step style into N = N1 * N2 (N1 >= N2):
//   input index  n = n1 + N1*n2,   output index k = k2 + N2*k1,
//   X[k2 + N2 k1] = sum_n1 W_N^{n1 k2} W_N1^{n1 k1} sum_n2 x[n1 + N1 n2] W_N2^{n2 k2}.
// Step A: one thread per (signal, n1) does the N2-point DFT in registers and the
// twiddle; step B: one thread per (signal, k2) does the N1-point DFT of a
// contiguous row. Both steps work in place; afterwards X[k] sits at position
// k1 + N1*k2. One padding element after every N1 keeps both steps free of shared-
// memory bank conflicts.
#pragma once

#include "common.cuh"

namespace cg {

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

__host__ __device__ constexpr int bitrev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((x >> i) & 1);
  return r;
}

// In-register DFT of R (power of two) points. W[p] = exp(s 2 pi i p / N) is the root
// table of the enclosing length-N transform (the sign s picks the direction);
// tstride = N / R. Radix-2 decimation in time after a compile-time bit reversal.
template <typename C, int R>
__device__ __forceinline__ void reg_dft(C (&a)[R], const C* __restrict__ W, int tstride) {
  constexpr int LR = ilog2c(R);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = bitrev(i, LR);
    if (j > i) {
      C t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
#pragma unroll
  for (int half = 1; half < R; half <<= 1) {
#pragma unroll
    for (int i = 0; i < R; i += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        C v = a[i + j + half];
        if (j != 0) v = cmul(v, W[j * (R / (2 * half)) * tstride]);
        const C u = a[i + j];
        a[i + j] = cadd(u, v);
        a[i + j + half] = csub(u, v);
      }
    }
  }
}

template <int LOG2N>
struct FFTShape {
  static constexpr int N = 1 << LOG2N;
  static constexpr int L1 = (LOG2N + 1) / 2;
  static constexpr int L2 = LOG2N - L1;
  static constexpr int N1 = 1 << L1;   // length of the step-B DFTs (rows)
  static constexpr int N2 = 1 << L2;   // length of the step-A DFTs (columns)
  static constexpr int STRIDE = N + N / N1;  // padded length of one signal in shared memory
  static constexpr int SSTRIDE = STRIDE + 1; // distance between signals (shifts their banks)
  __device__ static __forceinline__ int pidx(int p) { return p + (p >> L1); }
  // shared-memory slot of output X[k] once block_fft has run
  __device__ static __forceinline__ int out_slot(int k) {
    return pidx((k >> L2) + N1 * (k & (N2 - 1)));
  }
};

// In-place DFT of S signals stored at buf[s*SSTRIDE + pidx(p)], p in [0, N), with root
// table W (shared memory, N entries). Unnormalised. Ends with __syncthreads().
template <typename T, int LOG2N>
__device__ __forceinline__ void block_fft(V2<T>* buf, int S, const V2<T>* __restrict__ W) {
  using C = V2<T>;
  using F = FFTShape<LOG2N>;
  for (int task = threadIdx.x; task < S * F::N1; task += blockDim.x) {
    const int s = task >> F::L1, n1 = task & (F::N1 - 1);
    C* x = buf + s * F::SSTRIDE;
    C a[F::N2];
#pragma unroll
    for (int n2 = 0; n2 < F::N2; ++n2) a[n2] = x[F::pidx(n1 + F::N1 * n2)];
    reg_dft<C, F::N2>(a, W, F::N1);
#pragma unroll
    for (int k2 = 1; k2 < F::N2; ++k2) a[k2] = cmul(a[k2], W[n1 * k2]);
#pragma unroll
    for (int k2 = 0; k2 < F::N2; ++k2) x[F::pidx(n1 + F::N1 * k2)] = a[k2];
  }
  __syncthreads();
  for (int task = threadIdx.x; task < S * F::N2; task += blockDim.x) {
    const int s = task >> F::L2, k2 = task & (F::N2 - 1);
    C* x = buf + s * F::SSTRIDE;
    C a[F::N1];
#pragma unroll
    for (int n1 = 0; n1 < F::N1; ++n1) a[n1] = x[F::pidx(n1 + F::N1 * k2)];
    reg_dft<C, F::N1>(a, W, F::N2);
#pragma unroll
    for (int k1 = 0; k1 < F::N1; ++k1) x[F::pidx(k1 + F::N1 * k2)] = a[k1];
  }
  __syncthreads();
}

}  // namespace cg
