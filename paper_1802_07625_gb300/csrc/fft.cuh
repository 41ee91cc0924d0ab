// Shared-memory batched complex FFT for power-of-two lengths 8..1024.
//
// A length-N transform is split four-step style into N = N1 * N2 (N1 >= N2):
//   input index  n = n1 + N1*n2,   output index k = k2 + N2*k1,
//   X[k2 + N2 k1] = sum_n1 W_N^{n1 k2} W_N1^{n1 k1} sum_n2 x[n1 + N1 n2] W_N2^{n2 k2}.
// Step A: one thread per (signal, n1) does the N2-point DFT in registers and the
// twiddle W_N^{n1 k2}; step B: one thread per (signal, k2) does the N1-point DFT of a
// contiguous row. Both steps work in place; afterwards X[k] sits at position
// k1 + N1*k2. One padding element after every N1 keeps both steps free of shared-
// memory bank conflicts.
//
// The register DFTs are radix-2 decimation in time with every twiddle a compile-time
// constant: cos and sin of 2 pi j / n are evaluated at compile time from their Taylor
// series after an exact integer reduction to the first quadrant; multiplications by
// 1 and by +-i are elided, and the other butterflies take their sum and difference by
// fused multiply-adds (u + w v directly, u - w v as 2u - (u + w v)).
#pragma once

#include <type_traits>
#include <utility>

#include "common.cuh"

namespace cg {

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

__host__ __device__ constexpr int bitrev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((x >> i) & 1);
  return r;
}

// Taylor series of sin and cos, accurate to double rounding on [0, pi/2].
__host__ __device__ constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int k = 1; k < 24; ++k) {
    t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k < 24; ++k) {
    t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}
// cos and sin of 2 pi k / n for n a multiple of 4: quadrant q = floor(4k/n) and
// remainder r = k - q n/4 are exact integers; x = 2 pi r / n lies in [0, pi/2).
__host__ __device__ constexpr double cos2pi(int k, int n) {
  const int kk = ((k % n) + n) % n;
  const int q = (4 * kk) / n, r = kk - q * (n / 4);
  const double x = 2.0 * 3.14159265358979323846 * r / n;
  return q == 0 ? taylor_cos(x) : q == 1 ? -taylor_sin(x) : q == 2 ? -taylor_cos(x) : taylor_sin(x);
}
__host__ __device__ constexpr double sin2pi(int k, int n) {
  const int kk = ((k % n) + n) % n;
  const int q = (4 * kk) / n, r = kk - q * (n / 4);
  const double x = 2.0 * 3.14159265358979323846 * r / n;
  return q == 0 ? taylor_sin(x) : q == 1 ? taylor_cos(x) : q == 2 ? -taylor_sin(x) : -taylor_cos(x);
}

// One radix-2 butterfly of a length-2*HALF sub-transform on a[U], a[U+HALF] with twiddle
// exp(s 2 pi i J / (2 HALF)), s = +1 for the inverse direction.
template <typename C, int R, bool INV, int HALF, int U, int J>
__device__ __forceinline__ void butterfly(C (&a)[R]) {
  using T = decltype(a[0].x);
  C v = a[U + HALF];
  if constexpr (J != 0) {
    if constexpr (4 * J == 2 * HALF) {
      // multiply by +i (inverse) or -i (forward)
      v = INV ? mk2<T>(-v.y, v.x) : mk2<T>(v.y, -v.x);
    } else if constexpr (std::is_same<T, float>::value || std::is_same<T, double>::value) {
      // u + w v by two fused multiply-adds per component, u - w v as 2u - (u + w v):
      // six instructions instead of a complex product and two complex additions
      constexpr double wr = cos2pi(J, 2 * HALF);
      constexpr double wi = (INV ? 1.0 : -1.0) * sin2pi(J, 2 * HALF);
      const T r = (T)wr, i = (T)wi;
      const C u = a[U];
      const T px = fma(-v.y, i, fma(v.x, r, u.x));
      const T py = fma(v.y, r, fma(v.x, i, u.y));
      a[U] = mk2<T>(px, py);
      a[U + HALF] = mk2<T>(fma(T(2), u.x, -px), fma(T(2), u.y, -py));
      return;
    } else {
      constexpr double wr = cos2pi(J, 2 * HALF);
      constexpr double wi = (INV ? 1.0 : -1.0) * sin2pi(J, 2 * HALF);
      const T r = (T)wr, i = (T)wi;
      v = mk2<T>(v.x * r - v.y * i, v.x * i + v.y * r);
    }
  }
  const C u = a[U];
  a[U] = cadd(u, v);
  a[U + HALF] = csub(u, v);
}

template <typename C, int R, bool INV, int HALF, int... B>
__device__ __forceinline__ void dft_stage(C (&a)[R], std::integer_sequence<int, B...>) {
  (butterfly<C, R, INV, HALF, (B / HALF) * 2 * HALF + (B % HALF), B % HALF>(a), ...);
}

template <typename C, int R, int I>
__device__ __forceinline__ void bitrev_swap(C (&a)[R]) {
  constexpr int J = bitrev(I, ilog2c(R));
  if constexpr (J > I) {
    const C t = a[I];
    a[I] = a[J];
    a[J] = t;
  }
}
template <typename C, int R, int... I>
__device__ __forceinline__ void bitrev_all(C (&a)[R], std::integer_sequence<int, I...>) {
  (bitrev_swap<C, R, I>(a), ...);
}

template <typename C, int R, bool INV, int HALF>
__device__ __forceinline__ void dft_stages(C (&a)[R]) {
  if constexpr (HALF < R) {
    dft_stage<C, R, INV, HALF>(a, std::make_integer_sequence<int, R / 2>{});
    dft_stages<C, R, INV, 2 * HALF>(a);
  }
}

// In-register unnormalised DFT of R points (power of two), direction INV.
template <typename C, int R, bool INV>
__device__ __forceinline__ void reg_dft(C (&a)[R]) {
  if constexpr (R > 1) {
    bitrev_all<C, R>(a, std::make_integer_sequence<int, R>{});
    dft_stages<C, R, INV, 1>(a);
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

// DFT of S signals into buf[s*SSTRIDE + pidx(p)], p in [0, N): step A takes its inputs
// from load(s, n1, a), which fills a[n2] with element n1 + N1*n2 of signal s (so a pass can
// form its signals on the fly instead of staging them in buf first), and leaves its results
// in buf, where step B finishes in place. TW[k2*N1 + n1] = exp(s 2 pi i n1 k2 / N) holds the
// inter-step twiddles (shared memory; consecutive threads read consecutive entries).
// Unnormalised. Ends with __syncthreads().
template <typename T, int LOG2N, bool INV, typename Load>
__device__ __forceinline__ void block_fft_from(V2<T>* buf, int S, const V2<T>* __restrict__ TW, Load&& load) {
  using C = V2<T>;
  using F = FFTShape<LOG2N>;
  for (int task = threadIdx.x; task < S * F::N1; task += blockDim.x) {
    const int s = task >> F::L1, n1 = task & (F::N1 - 1);
    C* x = buf + s * F::SSTRIDE;
    C a[F::N2];
    load(s, n1, a);
    reg_dft<C, F::N2, INV>(a);
#pragma unroll
    for (int k2 = 1; k2 < F::N2; ++k2) a[k2] = cmul(a[k2], TW[k2 * F::N1 + n1]);
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
    reg_dft<C, F::N1, INV>(a);
#pragma unroll
    for (int k1 = 0; k1 < F::N1; ++k1) x[F::pidx(k1 + F::N1 * k2)] = a[k1];
  }
  __syncthreads();
}

// In-place DFT of S signals stored at buf[s*SSTRIDE + pidx(p)], p in [0, N) (see
// block_fft_from). Ends with __syncthreads().
// COMPACT (where N1 = N2): both steps run one copy of the register DFT in a loop over the
// two steps, with the element positions n + N1 k (step A) or N1 n + k (step B) taken at run
// time: the same arithmetic in the same order, in half the code. For the float-float type,
// whose unrolled register DFT is large, the two inlined copies overflow the instruction
// cache.
template <typename T, int LOG2N, bool INV, bool COMPACT = false>
__device__ __forceinline__ void block_fft(V2<T>* buf, int S, const V2<T>* __restrict__ TW) {
  using C = V2<T>;
  using F = FFTShape<LOG2N>;
  if constexpr (COMPACT && F::N1 == F::N2) {
#pragma unroll 1
    for (int step = 0; step < 2; ++step) {
      for (int task = threadIdx.x; task < S * F::N1; task += blockDim.x) {
        const int s = task >> F::L1, n = task & (F::N1 - 1);
        C* x = buf + s * F::SSTRIDE;
        const int base = step ? F::N1 * n : n, stride = step ? 1 : F::N1;
        C a[F::N1];
#pragma unroll
        for (int k = 0; k < F::N1; ++k) a[k] = x[F::pidx(base + stride * k)];
        reg_dft<C, F::N1, INV>(a);
        if (step == 0) {
#pragma unroll
          for (int k2 = 1; k2 < F::N2; ++k2) a[k2] = cmul(a[k2], TW[k2 * F::N1 + n]);
        }
#pragma unroll
        for (int k = 0; k < F::N1; ++k) x[F::pidx(base + stride * k)] = a[k];
      }
      __syncthreads();
    }
  } else {
    block_fft_from<T, LOG2N, INV>(buf, S, TW, [&](int s, int n1, C (&a)[F::N2]) {
      const C* x = buf + s * F::SSTRIDE;
#pragma unroll
      for (int n2 = 0; n2 < F::N2; ++n2) a[n2] = x[F::pidx(n1 + F::N1 * n2)];
    });
  }
}

}  // namespace cg
