// Spectral kernels of the diffusion flow.
//
// Forward: the cosine transform of the normalised, mean-subtracted density with the
// blur factor (main text Eq. rhotilde_mn; SI Eq. rhoxyt's coefficients), computed as
// a DCT-II along x then along y, each through one complex FFT per pair of real lines.
//
// Inverse (every attempted step): SI Eq. rhoxyt with f_mn = exp(-pi^2 (m^2/Lx^2 +
// n^2/Ly^2) t) (Eq. fmn_diff, D = 1) and its x and y derivatives. The damping is
// separable, exp(-pi^2 m^2 t/Lx^2) exp(-pi^2 n^2 t/Ly^2), so each block evaluates
// Lx + (rows) exponentials instead of one per coefficient.
//   pass 1 (rows n, along x):  A[n][i] = sum_m a_nm cos(pi m x_i/Lx)
//                              B[n][i] = sum_m a_nm (-pi m/Lx) sin(pi m x_i/Lx)
//   pass 2 (columns i, along y): rho' = sum_n A cos,  d_y rho = sum_n A (-pi n/Ly) sin,
//                              d_x rho = sum_n B cos;  v = -grad rho / (1 + rho')
// A length-N cosine sum y_i = sum_m c_m cos(pi m (i+1/2)/N) is one complex inverse DFT
// of U_m = e^{i pi m/(2N)} (c_m - i c_{N-m})/2 (U_0 = c_0) read back in the order
// y_{2k} = u_k, y_{2k+1} = u_{N-1-k}; a sine sum is the cosine sum of the reversed
// coefficients times (-1)^i. Two real sums share one complex DFT (real and imaginary
// parts).
#pragma once

#include <type_traits>

#include "fft.cuh"
#include "tma.cuh"

namespace cg {

__device__ __forceinline__ float texp(float x) { return expf(x); }
__device__ __forceinline__ double texp(double x) { return exp(x); }

// Two adjacent outputs with one store where the pair is one aligned vector (the callers'
// pairs start at even indices of arrays that start at 16-byte boundaries).
__device__ __forceinline__ void st_two(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_two(double2* p, double2 a, double2 b) {
  p[0] = a;
  p[1] = b;
}
__device__ __forceinline__ void st_two(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ void st_two(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

// a * b + c, with one rounding in FP32 and FP64
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return fma(a, b, c); }
template <typename A> __device__ __forceinline__ A madd(A a, A b, A c) { return a * b + c; }

// 1 / x of the velocity v = -grad rho / rho. In FP32 the hardware's approximate reciprocal
// (within 2 ulp for the positive normal densities here, far inside the error of the FP32
// transforms that produce rho); in FP64 and float-float a division.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
template <typename A> __device__ __forceinline__ A recip(A x) { return A(1) / x; }

// Output index i of a cosine sum -> index of the complex DFT output that holds it.
__device__ __forceinline__ int dct3_src(int i, int N) { return (i & 1) ? (N - 1 - (i >> 1)) : (i >> 1); }

// Shared-memory footprint (bytes) of one pass-1 item of S rows and one pass-2 item of
// Wc columns; mirrored by the host-side launch configurations.
template <typename T, int LOG2N>
__host__ __device__ constexpr size_t p1_smem(int S) {
  using F = FFTShape<LOG2N>;
  return (size_t)F::N * 4 * sizeof(T) + (size_t)S * F::N * sizeof(T) +
         (size_t)S * F::SSTRIDE * 2 * sizeof(T) + (size_t)(F::N + S) * sizeof(T);
}
// Pass 2 stages its columns and quarter-wave factors in shared memory except in FP64, whose
// 16-byte elements would leave one block (three warps) per SM: there it reads both from
// global memory (L2 and L1) and fits three blocks per SM.
template <typename T> __host__ __device__ constexpr bool p2_staged() { return !std::is_same<T, double>::value; }
template <typename T, int LOG2N, typename A = T>
__host__ __device__ constexpr size_t p2_smem(int Wc) {
  using F = FFTShape<LOG2N>;
  return p2_staged<T>()
             ? (size_t)F::N * 4 * sizeof(A) + (size_t)Wc * F::N * 2 * sizeof(T) +
                   (size_t)(Wc + Wc / 2) * F::SSTRIDE * 2 * sizeof(A) + 64 * sizeof(T)
             : (size_t)F::N * 2 * sizeof(A) + (size_t)(Wc + Wc / 2) * F::SSTRIDE * 2 * sizeof(A) + 64 * sizeof(T);
}

// A read-only table entry.
template <typename C> __device__ __forceinline__ C ld_table(const C* p) { return __ldg(p); }

// Issue the bulk copies of a pass-1 item (thread 0): both tables and the S spectral rows,
// none of which depend on the previous kernel of the step loop.
template <typename T, int LOG2N>
__device__ __forceinline__ void p1_issue(const T* __restrict__ spec, const V2<T>* __restrict__ Wg,
                                         const V2<T>* __restrict__ Eg, int S, int n0,
                                         unsigned char* smem, uint64_t* bar) {
  using C = V2<T>;
  constexpr int N = 1 << LOG2N;
  C* W = reinterpret_cast<C*>(smem);
  C* E = W + N;
  T* stage = reinterpret_cast<T*>(E + N);
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    mbar_expect_tx(bar, (uint32_t)(2 * N * sizeof(C) + S * N * sizeof(T)));
    bulk_g2s(W, Wg, N * sizeof(C), bar);
    bulk_g2s(E, Eg, N * sizeof(C), bar);
    for (int s = 0; s < S; ++s) bulk_g2s(stage + s * N, spec + (size_t)(n0 + s) * N, N * sizeof(T), bar);
  }
}

// Damping rates of the diffusion time tau in the working type: kx = pi^2 tau / Lx^2,
// ky = pi^2 tau / Ly^2 (Lx = 2^LOG2N).
// The divisions by the squared sizes (powers of two) are exact, so they are taken as
// multiplications by the exact reciprocals (FP64 division is slow on GB300).
template <typename T, int LOG2N>
__device__ __forceinline__ void damp_rates(double tau, int Ly, T& kx, T& ky) {
  const double pt = kPi * kPi * tau;
  const int log2Ly = __ffs(Ly) - 1;
  kx = (T)(pt * __longlong_as_double((long long)(1023 - 2 * LOG2N) << 52));
  ky = (T)(pt * __longlong_as_double((long long)(1023 - 2 * log2Ly) << 52));
}

// Rest of a pass-1 item once its copies are issued: damping with the rates kx, ky
// (damp_rates), packing, FFT, transposed write. All threads call it; false if the
// copies did not complete.
template <typename T, int LOG2N>
__device__ __forceinline__ bool p1_finish(V2<T>* __restrict__ ABt, int Ly, int S, int n0, T kx, T ky,
                                          unsigned char* smem, uint64_t* bar, uint32_t& ph) {
  using C = V2<T>;
  using F = FFTShape<LOG2N>;
  constexpr int N = F::N;
  C* W = reinterpret_cast<C*>(smem);
  C* E = W + N;
  T* stage = reinterpret_cast<T*>(E + N);
  C* buf = reinterpret_cast<C*>(stage + S * N);
  T* fx = reinterpret_cast<T*>(buf + S * F::SSTRIDE);
  T* fyS = fx + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) fx[i] = texp(-kx * (T)i * (T)i) / (T)N;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const T n = (T)(n0 + s);
    fyS[s] = texp(-ky * n * n) / (T)Ly;
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(bar, ph, kMbarTries);
  ph ^= 1u;
  if (!__syncthreads_and(ok)) return false;

  const T kd = (T)(kPi / N);
  // The packed signal of each row, formed by the FFT's first step as it reads its inputs
  // (no staging pass): element m > 0 of row s is E[m] ((a_m + b_m)/2, (b_q - a_q)/2), q = N - m,
  // with a_m = spec[m] fx[m] fy and b_m = -(pi m / N) a_m (the DCT-III and DST-III
  // coefficients sharing one complex DFT); element 0 is (a_0, 0).
  block_fft_from<T, LOG2N, true>(buf, S, W, [&](int s, int n1, C (&a)[F::N2]) {
    const T* row = stage + s * N;
    const T f = fyS[s];
    const T fn1 = (T)n1;  // m and N - m as values by exact adds, not a conversion each
#pragma unroll
    for (int n2 = 0; n2 < F::N2; ++n2) {
      const int m = n1 + F::N1 * n2, q = (N - m) & (N - 1);
      const T fm = fn1 + T(F::N1 * n2), fq = T(N) - fm;
      const T am = row[m] * fx[m] * f;
      const T aq = row[q] * fx[q] * f;
      const T bm = -kd * fm * am;
      const T bq = -kd * fq * aq;
      a[n2] = (m == 0) ? mk2<T>(am, T(0)) : cmul(E[m], mk2<T>((am + bm) * T(0.5), (bq - aq) * T(0.5)));
    }
  });
  // S is a power of two: a runtime integer division here costs as much as the FFT. Two
  // adjacent rows per task (one output slot, one vector store)
  const int ls = __ffs(S) - 1;
  if (S >= 2) {
    for (int task = threadIdx.x; task < (S * N) >> 1; task += blockDim.x) {
      const int i = task >> (ls - 1), s = 2 * (task & ((S >> 1) - 1));
      const int slot = F::out_slot(dct3_src(i, N));
      const C ua = buf[s * F::SSTRIDE + slot], ub = buf[(s + 1) * F::SSTRIDE + slot];
      st_two(ABt + (size_t)i * Ly + n0 + s, mk2<T>(ua.x, (i & 1) ? -ua.y : ua.y), mk2<T>(ub.x, (i & 1) ? -ub.y : ub.y));
    }
  } else {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const C u = buf[F::out_slot(dct3_src(i, N))];
      ABt[(size_t)i * Ly + n0] = mk2<T>(u.x, (i & 1) ? -u.y : u.y);
    }
  }
  __syncthreads();
  return true;
}

// pass 1 item: damped spectrum rows [n0, n0+S) -> (A, B), written transposed: ABt[i][n].
// The tables and the S spectral rows arrive in shared memory by bulk asynchronous
// copies on `bar` (phase `ph`, toggled here) while the damping factors are computed.
// shared: W[N] (inter-step twiddles) E[N] (C), stage[S*N] (T), buf[S*SSTRIDE] (C),
// fx[N] fy[S] (T)
template <typename T, int LOG2N>
__device__ __forceinline__ bool p1_rows(const T* __restrict__ spec, V2<T>* __restrict__ ABt,
                                        const V2<T>* __restrict__ Wg, const V2<T>* __restrict__ Eg,
                                        int Ly, int S, int n0, double tau, unsigned char* smem,
                                        uint64_t* bar, uint32_t& ph) {
  p1_issue<T, LOG2N>(spec, Wg, Eg, S, n0, smem, bar);
  T kx, ky;
  damp_rates<T, LOG2N>(tau, Ly, kx, ky);
  return p1_finish<T, LOG2N>(ABt, Ly, S, n0, kx, ky, smem, bar, ph);
}

// A complex value in the arithmetic type A.
template <typename A, typename T> __device__ __forceinline__ V2<A> to_v2(const V2<T>& v) {
  return mk2<A>(A(v.x), A(v.y));
}

// Block-reduced results of a pass-2 item (valid in thread 0).
template <typename T> struct FieldRed {
  T dev;    // max |rho/rho_bar - 1|
  T v2max;  // max |v|^2
  bool bad; // a non-positive or non-finite density
};

// ---------------------------------------------------------------------------
// pass 2 item: (A, B) columns [c0, c0+Wc) -> velocity (Wc even): Wc signals for
// (rho', d_y rho) and Wc/2 signals for d_x rho of column pairs. The Wc columns of ABt
// are contiguous and arrive with the tables by bulk asynchronous copies.
// shared: W[N] E[N] (C), stage[Wc*N] (C), buf[(Wc + Wc/2) * SSTRIDE] (C), red[64] (T)
// ---------------------------------------------------------------------------
// Pass-2 copies in two parts on one mbarrier phase (thread 0): the tables, which do not
// depend on pass 1, and then the Wc columns of ABt that pass 1 wrote.
template <typename T, int LOG2N, typename A = T>
__device__ __forceinline__ void p2_issue_tables(const V2<A>* __restrict__ Wg, const V2<A>* __restrict__ Eg,
                                                int Wc, unsigned char* smem, uint64_t* bar) {
  using C = V2<A>;
  constexpr int N = 1 << LOG2N;
  C* W = reinterpret_cast<C*>(smem);
  C* E = W + N;
  if (threadIdx.x == 0) {
    if constexpr (p2_staged<T>()) {
      mbar_expect_tx(bar, (uint32_t)(2 * N * sizeof(C) + Wc * N * sizeof(V2<T>)));
      bulk_g2s(W, Wg, N * sizeof(C), bar);
      bulk_g2s(E, Eg, N * sizeof(C), bar);
    } else {
      mbar_expect_tx(bar, (uint32_t)(N * sizeof(C)));
      bulk_g2s(W, Wg, N * sizeof(C), bar);
    }
  }
}
template <typename T, int LOG2N, typename A = T>
__device__ __forceinline__ void p2_issue_cols(const V2<T>* __restrict__ ABt, int Wc, int c0,
                                              unsigned char* smem, uint64_t* bar) {
  using C = V2<T>;
  constexpr int N = 1 << LOG2N;
  C* stage = reinterpret_cast<C*>(reinterpret_cast<V2<A>*>(smem) + 2 * N);
  if constexpr (!p2_staged<T>()) return;  // read in place by p2_finish
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    for (int cc = 0; cc < Wc; ++cc)
      bulk_g2s(stage + cc * N, ABt + (size_t)(c0 + cc) * N, N * sizeof(C), bar);
  }
}

// ---------------------------------------------------------------------------
// pass 2 item: (A, B) columns [c0, c0+Wc) -> velocity (Wc even): Wc signals for
// (rho', d_y rho) and Wc/2 signals for d_x rho of column pairs, once the copies issued
// by p2_issue_tables and p2_issue_cols have landed.
// shared: W[N] E[N] (C), stage[Wc*N] (C), buf[(Wc + Wc/2) * SSTRIDE] (C), red[64] (T)
// ---------------------------------------------------------------------------
// T: the type of the (A, B) input, of the field written and of the reductions; A: the
// arithmetic of the packing, the FFT and the velocity (T, or float-float for FP32 data).
// ABt and Eg: the columns and the quarter-wave factors in global memory, read there where
// pass 2 does not stage them (p2_staged).
template <typename T, int LOG2N, typename A = T>
__device__ __forceinline__ bool p2_finish(V2<T>* __restrict__ out, T* __restrict__ rho_out, int Lx,
                                          int Wc, int c0, unsigned char* smem, uint64_t* bar,
                                          uint32_t& ph, FieldRed<T>& res, bool raw,
                                          const V2<T>* __restrict__ ABt, const V2<A>* __restrict__ Eg) {
  using C = V2<A>;
  using F = FFTShape<LOG2N>;
  constexpr int N = F::N;  // = Ly
  constexpr bool kStaged = p2_staged<T>();
  C* W = reinterpret_cast<C*>(smem);
  C* E = W + N;
  const V2<T>* stage = kStaged ? reinterpret_cast<const V2<T>*>(E + N) : ABt + (size_t)c0 * N;
  C* buf = kStaged ? reinterpret_cast<C*>(reinterpret_cast<V2<T>*>(E + N) + Wc * N) : E;
  T* red = reinterpret_cast<T*>(buf + (Wc + Wc / 2) * F::SSTRIDE);
  auto ld_in = [&](const V2<T>* p) -> C {
    if constexpr (kStaged) return to_v2<A, T>(*p);
    else return to_v2<A, T>(__ldcg(p));  // written by pass 1 (L2)
  };
  auto ld_e = [&](int m) -> C {
    if constexpr (kStaged) return E[m];
    else return ld_table(Eg + m);
  };
  const bool ok = mbar_wait_bounded(bar, ph, kMbarTries);
  ph ^= 1u;
  if (!__syncthreads_and(ok)) return false;

  const int Wp = Wc / 2;
  const A kh = (A)(0.5 * kPi / N);
  // N/2 tasks per column pair (no runtime integer division): task m > 0 packs the pair
  // (m, N - m); task 0 packs m = 0 and then (second round) the self-paired m = N/2.
  // With b_m = -(pi m/N) a_m, (a_m + b_m)/2 = a_m g_m and (b_m - a_m)/2 = a_m h_m, where
  // g_m = 1/2 - (pi/(2N)) m and h_m = -1/2 - (pi/(2N)) m.
  for (int task = threadIdx.x; task < (N / 2) * Wp; task += blockDim.x) {
    const int p = task >> (LOG2N - 1);
    int m = task & (N / 2 - 1);
    const V2<T>* s0 = stage + (2 * p) * N;
    const V2<T>* s1 = s0 + N;
    C* x0 = buf + (2 * p) * F::SSTRIDE;
    C* x1 = x0 + F::SSTRIDE;
    C* x2 = buf + (Wc + p) * F::SSTRIDE;
    if (m == 0) {
      const C A00 = ld_in(s0), A01 = ld_in(s1);
      x0[F::pidx(0)] = mk2<A>(A00.x, A(0));
      x1[F::pidx(0)] = mk2<A>(A01.x, A(0));
      x2[F::pidx(0)] = mk2<A>(A00.y, A01.y);
      m = N / 2;
    }
    const C Am0 = ld_in(s0 + m), Am1 = ld_in(s1 + m);
    const int q = N - m;
    const C Aq0 = ld_in(s0 + q), Aq1 = ld_in(s1 + q);
    const C em = ld_e(m), eq = ld_e(q);
    const A fm = int_to(m, A(0)), fq = A(N) - fm;
    const A gm = madd(-kh, fm, A(0.5)), hm = madd(-kh, fm, A(-0.5));
    const A gq = madd(-kh, fq, A(0.5)), hq = madd(-kh, fq, A(-0.5));
    {  // (rho', d_y rho) of column c
      const A am = Am0.x, aq = Aq0.x;
      x0[F::pidx(m)] = cmul(em, mk2<A>(am * gm, aq * hq));
      if (q != m) x0[F::pidx(q)] = cmul(eq, mk2<A>(aq * gq, am * hm));
    }
    {  // (rho', d_y rho) of column c + 1
      const A am = Am1.x, aq = Aq1.x;
      x1[F::pidx(m)] = cmul(em, mk2<A>(am * gm, aq * hq));
      if (q != m) x1[F::pidx(q)] = cmul(eq, mk2<A>(aq * gq, am * hm));
    }
    {  // d_x rho of columns c (real part) and c + 1 (imaginary part)
      const A bem = Am0.y, gam = Am1.y, beq = Aq0.y, gaq = Aq1.y;
      x2[F::pidx(m)] = cmul(em, mk2<A>((bem + gaq) * A(0.5), (gam - beq) * A(0.5)));
      if (q != m) x2[F::pidx(q)] = cmul(eq, mk2<A>((beq + gam) * A(0.5), (gaq - bem) * A(0.5)));
    }
  }
  __syncthreads();
  block_fft<A, LOG2N, true, !std::is_same<A, T>::value>(buf, Wc + Wp, W);

  T dev = T(0), v2max = T(0);
  bool bad = false;
  // a column pair per task (Wc is an even power of two; no runtime integer division): the
  // two columns share the output slot and the d_x rho signal (real and imaginary parts)
  const int lp = __ffs(Wc) - 2;
  for (int task = threadIdx.x; task < (N * Wc) >> 1; task += blockDim.x) {
    const int j = task >> lp, cp = task & ((Wc >> 1) - 1);
    const int slot = F::out_slot(dct3_src(j, N));
    const C u2 = buf[(Wc + cp) * F::SSTRIDE + slot];
    V2<T> vv[2];
    T rr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const C u1 = buf[(2 * cp + h) * F::SSTRIDE + slot];
      const A rp = u1.x;
      const A gy = (j & 1) ? -u1.y : u1.y;
      const A gx = h ? u2.y : u2.x;
      const A rho = A(1) + rp;
      if (!raw) bad |= !(rho > A(0));
      const A inv = raw ? A(1) : recip(rho);
      const T vx = (T)(-gx * inv), vy = (T)(-gy * inv);
      vv[h] = mk2<T>(vx, vy);
      rr[h] = (T)(raw ? rp : rho);  // flux mode: the plain cosine sum
      dev = max(dev, fabs((T)rp));
      v2max = max(v2max, vx * vx + vy * vy);
    }
    const size_t o = (size_t)j * Lx + c0 + 2 * cp;
    st_two(out + o, vv[0], vv[1]);
    if (rho_out) st_two(rho_out + o, rr[0], rr[1]);
  }
  // both maxima and the flag with one barrier (valid in thread 0)
  dev = warp_max(dev);
  v2max = warp_max(v2max);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp] = dev;
    red[32 + warp] = v2max;
  }
  res.bad = __syncthreads_or(bad);
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    dev = warp_max(lane < nw ? red[lane] : T(0));
    v2max = warp_max(lane < nw ? red[32 + lane] : T(0));
  }
  res.dev = dev;
  res.v2max = v2max;
  __syncthreads();
  return true;
}

template <typename T, int LOG2N>
__device__ __forceinline__ bool p2_cols(const V2<T>* __restrict__ ABt, V2<T>* __restrict__ out,
                                        T* __restrict__ rho_out, const V2<T>* __restrict__ Wg,
                                        const V2<T>* __restrict__ Eg, int Lx, int Wc, int c0,
                                        unsigned char* smem, uint64_t* bar, uint32_t& ph,
                                        FieldRed<T>& res) {
  p2_issue_tables<T, LOG2N>(Wg, Eg, Wc, smem, bar);
  p2_issue_cols<T, LOG2N>(ABt, Wc, c0, smem, bar);
  return p2_finish<T, LOG2N>(out, rho_out, Lx, Wc, c0, smem, bar, ph, res, false, ABt, Eg);
}

// Programmatic dependent launch: let the next kernel of the step loop start its
// independent prologue, and wait for the previous kernel before using its results.
// Both are no-ops for a kernel launched without the programmatic-serialisation attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// pass 1 as its own kernel. blockDim = S * N1, grid = Ly / S. The bulk copies of the
// constant inputs (tables, spectral rows) start before waiting for the previous kernel.
// ---------------------------------------------------------------------------
template <typename T, int LOG2N>
__global__ void inv_rows_kernel(const T* __restrict__ spec, V2<T>* __restrict__ ABt,
                                const V2<T>* __restrict__ Wg, const V2<T>* __restrict__ Eg,
                                int Ly, int S, DevState* st, int mode, double tau_fixed,
                                cudaGraphConditionalHandle handle, int use_cond,
                                unsigned int max_body) {
  __shared__ __align__(8) uint64_t bar;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  p1_issue<T, LOG2N>(spec, Wg, Eg, S, blockIdx.x * S, smem_raw, &bar);
  __shared__ T s_k[2];
  __shared__ int s_run;
  pdl_wait();
  // thread 0 takes the attempt's time and the damping rates (FP64 arithmetic, once per
  // block: GB300's FP64 pipe is narrow)
  if (threadIdx.x == 0) {
    double tau = tau_fixed;
    int run = 1;
    if (is_step_mode(mode)) {
      // first kernel of an attempt: the controller's decision on the previous attempt
      // (every block computes it; block 0 stores it as this attempt's state, ends the
      // loop when the integration is over or has run more attempts than it allows, and
      // then also commits the final state)
      const int b = step_slot(mode);
      LoopSlot n = loop_decide(load_slot(&st->ls[b ^ 1]), load_sp(st), blockIdx.x == 0);
      if (blockIdx.x == 0) {
        const unsigned int it = atomicAdd(&st->body_iters, 1u) + 1u;
        if (n.status == kRunning && it > max_body) {
          n.status = kStepFail;
          n.pending = 0;
        }
        // every field but `bad`, which another block may already have flagged (it is
        // zero in a slot whose attempt was followed by another)
        LoopSlot* q = &st->ls[b];
        q->t = n.t;
        q->h = n.h;
        q->vmax = n.vmax;
        q->accepted = n.accepted;
        q->rejected = n.rejected;
        q->parity = n.parity;
        q->status = n.status;
        q->pending = n.pending;
        q->err2_bits = 0;
        q->vmax2_bits = 0;
        q->dev_bits = 0;
        if (n.status != kRunning) {
          st->t = n.t;
          st->h = n.h;
          st->vmax = n.vmax;
          st->accepted = n.accepted;
          st->rejected = n.rejected;
          st->parity = n.parity;
          st->status = n.status;
          if (use_cond) cudaGraphSetConditional(handle, 0);
        }
      }
      run = n.status == kRunning;
      tau = n.t + n.h;
    } else if (mode == kModeInit) {
      run = st->status == kRunning;
      tau = st->t;
    }
    s_run = run;
    T kx, ky;
    damp_rates<T, LOG2N>(tau, Ly, kx, ky);
    s_k[0] = kx;
    s_k[1] = ky;
  }
  __syncthreads();
  if (!s_run) {
    mbar_wait_bounded(&bar, 0, kMbarTries);  // no copy may be left in flight
    return;
  }
  uint32_t ph = 0;
  if (!p1_finish<T, LOG2N>(ABt, Ly, S, blockIdx.x * S, s_k[0], s_k[1], smem_raw, &bar, ph) && threadIdx.x == 0) {
    if (is_step_mode(mode)) atomicOr(&st->ls[step_slot(mode)].bad, 1);
    else st->bad = 2;
  }
  pdl_trigger();
}

// ---------------------------------------------------------------------------
// pass 2 as its own kernel. blockDim = (Wc + Wc/2) * N1, grid = Lx / Wc. A: the arithmetic
// (T, or float-float for FP32 data: the compensated mixed precision).
// ---------------------------------------------------------------------------
template <typename T, int LOG2N, typename A = T>
__global__ void inv_cols_kernel(const V2<T>* __restrict__ ABt, V2<T>* vbuf0, V2<T>* vbuf1,
                                T* __restrict__ rho_out, const V2<A>* __restrict__ Wg,
                                const V2<A>* __restrict__ Eg, int Lx, int Wc, DevState* st,
                                int mode) {
  __shared__ __align__(8) uint64_t bar;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const int c0 = blockIdx.x * Wc;
  p2_issue_tables<T, LOG2N, A>(Wg, Eg, Wc, smem_raw, &bar);
  __shared__ int s_run, s_par;
  const bool step = is_step_mode(mode);
  pdl_wait();
  p2_issue_cols<T, LOG2N, A>(ABt, Wc, c0, smem_raw, &bar);
  if (step) {
    // the attempt's state, as pass 1 decided and stored it (read while the copies land)
    if (threadIdx.x == 0) {
      const LoopSlot* q = &st->ls[step_slot(mode)];
      s_run = __ldcg(&q->status) == kRunning;
      s_par = __ldcg(&q->parity);
    }
    __syncthreads();
  }
  if ((step && !s_run) || (mode == kModeInit && st->status != kRunning)) {
    mbar_wait_bounded(&bar, 0, kMbarTries);  // no copy may be left in flight
    return;
  }
  V2<T>* out = vbuf0;
  if (step) out = s_par ? vbuf0 : vbuf1;
  else if (mode == kModeInit) out = st->parity ? vbuf1 : vbuf0;
  uint32_t ph = 0;
  FieldRed<T> r;
  if (!p2_finish<T, LOG2N, A>(out, rho_out, Lx, Wc, c0, smem_raw, &bar, ph, r, mode == kModeFlux, ABt, Eg)) {
    if (threadIdx.x == 0) {
      if (step) atomicOr(&st->ls[step_slot(mode)].bad, 1);
      else st->bad = 2;
    }
    return;
  }
  if (threadIdx.x == 0) {
    if (step) {
      LoopSlot* q = &st->ls[step_slot(mode)];
      atomic_max_nonneg(&q->dev_bits, (double)r.dev);
      atomic_max_nonneg(&q->vmax2_bits, (double)r.v2max);
      if (r.bad) atomicOr(&q->bad, 1);
    } else {
      atomic_max_nonneg(&st->dev_bits, (double)r.dev);
      atomic_max_nonneg(&st->vmax2_bits, (double)r.v2max);
      if (r.bad) st->bad = 1;
    }
  }
  pdl_trigger();
}

// ---------------------------------------------------------------------------
// forward pass 1: DCT-II along x of row pairs. S rows per block (even),
// blockDim = (S/2) * N1, grid = Ly / S. R[j][m] = sum_i rho[j][i] cos(pi m x_i/Lx).
// The two real rows of a signal come out of its DFT V as R[m] = Re(conj(E[m]) (V[m] +
// conj V[N-m]) / 2) and Re(conj(E[m]) (V[m] - conj V[N-m]) / (2i)); outputs m and N - m
// share the sums and differences of V[m] and V[N-m], so one task forms both, with the halves
// folded into a per-block table E/2 (exact).
// shared: W[N] (C, forward roots), buf[(S/2) * STRIDE] (C), Eh[N] (C)
// ---------------------------------------------------------------------------
// A: the arithmetic (FP64, or float-float for the mixed precisions); input and output FP64.
template <int LOG2N, typename A = double>
__global__ void fwd_rows_kernel(const double* __restrict__ rho, double* __restrict__ R,
                                const V2<A>* __restrict__ Wg, const V2<A>* __restrict__ Eg,
                                int S) {
  using C = V2<A>;
  using F = FFTShape<LOG2N>;
  constexpr int N = F::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* W = reinterpret_cast<C*>(smem_raw);
  C* buf = W + N;
  const int r0 = blockIdx.x * S;
  const int S2 = S / 2;
  C* Eh = buf + S2 * F::SSTRIDE;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    W[i] = Wg[i];
    const C e = Eg[i];
    Eh[i] = mk2<A>(A(0.5) * e.x, A(0.5) * e.y);
  }
  for (int task = threadIdx.x; task < S2 * (N / 2); task += blockDim.x) {
    const int s = task / (N / 2), k = task - s * (N / 2);
    const double2 e = *reinterpret_cast<const double2*>(rho + (size_t)(r0 + 2 * s) * N + 2 * k);
    const double2 o = *reinterpret_cast<const double2*>(rho + (size_t)(r0 + 2 * s + 1) * N + 2 * k);
    C* x = buf + s * F::SSTRIDE;
    x[F::pidx(k)] = mk2<A>(A(e.x), A(o.x));
    x[F::pidx(N - 1 - k)] = mk2<A>(A(e.y), A(o.y));
  }
  __syncthreads();
  block_fft<A, LOG2N, false, !std::is_same<A, double>::value>(buf, S2, W);
  for (int task = threadIdx.x; task < S2 * (N / 2); task += blockDim.x) {
    const int s = task >> (LOG2N - 1), k = task & (N / 2 - 1);
    const C* x = buf + s * F::SSTRIDE;
    double* R0 = R + (size_t)(r0 + 2 * s) * N;
    double* R1 = R0 + N;
    if (k == 0) {
      // the self-paired outputs 0 and N/2 (E[0] = 1)
      const C V0 = x[F::out_slot(0)], Vh = x[F::out_slot(N / 2)];
      const A eh = Eh[N / 2].x;
      R0[0] = (double)V0.x;
      R1[0] = (double)V0.y;
      R0[N / 2] = (double)(eh * (Vh.x + Vh.x));
      R1[N / 2] = (double)(eh * (Vh.y + Vh.y));
    } else {
      const int q = N - k;
      const C Vm = x[F::out_slot(k)], Vq = x[F::out_slot(q)];
      const A u = Vm.x + Vq.x, v = Vm.y - Vq.y, w = Vm.y + Vq.y, z = Vm.x - Vq.x;
      const C em = Eh[k], eq = Eh[q];
      R0[k] = (double)(em.x * u + em.y * v);
      R1[k] = (double)(em.x * w - em.y * z);
      R0[q] = (double)(eq.x * u - eq.y * v);
      R1[q] = (double)(eq.x * w + eq.y * z);
    }
  }
}

// ---------------------------------------------------------------------------
// forward pass 2: DCT-II along y of column pairs, times the coefficient weights
// 4/((1+d_m0)(1+d_n0)) and the separable blur factors; the (0,0) coefficient (the
// mean, which the velocity handles separately) is set to zero.
// Wc columns per block (even), blockDim = (Wc/2) * N1, grid = Lx / Wc. As in pass 1 one task
// forms outputs n and N - n; the halves and the row weights (1 + d_n0)^-1 2 by[n] are folded
// into a per-block table Ew[n] = E[n] (n == 0 ? 1/2 : 1) by[n].
// shared: W[N] (C), buf[(Wc/2) * SSTRIDE] (C), Ew[N] (C)
// A: the arithmetic (FP64, or float-float for the mixed precisions); input and output FP64.
// ---------------------------------------------------------------------------
template <typename T, int LOG2N, typename A = double>
__global__ void fwd_cols_kernel(const double* __restrict__ R, double* __restrict__ spec64,
                                T* __restrict__ specT, const V2<A>* __restrict__ Wg,
                                const V2<A>* __restrict__ Eg, const double* __restrict__ bx,
                                const double* __restrict__ by, int Lx, int Wc) {
  using C = V2<A>;
  using F = FFTShape<LOG2N>;
  constexpr int N = F::N;  // = Ly
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* W = reinterpret_cast<C*>(smem_raw);
  C* buf = W + N;
  const int c0 = blockIdx.x * Wc;
  const int Wp = Wc / 2;
  const int lp = __ffs(Wp) - 1;  // Wp is a power of two
  C* Ew = buf + Wp * F::SSTRIDE;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    W[i] = Wg[i];
    const C e = Eg[i];
    const A f = A((i == 0 ? 0.5 : 1.0) * (by ? by[i] : 1.0));
    Ew[i] = mk2<A>(e.x * f, e.y * f);
  }
  for (int task = threadIdx.x; task < (N / 2) * Wp; task += blockDim.x) {
    const int k = task >> lp, p = task & (Wp - 1);
    const double2 e = *reinterpret_cast<const double2*>(R + (size_t)(2 * k) * Lx + c0 + 2 * p);
    const double2 o = *reinterpret_cast<const double2*>(R + (size_t)(2 * k + 1) * Lx + c0 + 2 * p);
    C* x = buf + p * F::SSTRIDE;
    x[F::pidx(k)] = mk2<A>(A(e.x), A(e.y));
    x[F::pidx(N - 1 - k)] = mk2<A>(A(o.x), A(o.y));
  }
  __syncthreads();
  block_fft<A, LOG2N, false, !std::is_same<A, double>::value>(buf, Wp, W);
  auto put = [&](int n, int m, A a0, A a1) {
    const double s0 = (double)a0, s1 = (double)a1;
    const size_t o = (size_t)n * Lx + m;
    spec64[o] = s0;
    spec64[o + 1] = s1;
    if (specT) {
      specT[o] = (T)s0;
      specT[o + 1] = (T)s1;
    }
  };
  for (int task = threadIdx.x; task < (N / 2) * Wp; task += blockDim.x) {
    const int k = task >> lp, p = task & (Wp - 1);
    const C* x = buf + p * F::SSTRIDE;
    const int m = c0 + 2 * p;
    // column weights (1 + d_m0)^-1 2 bx[m]
    const A wm0 = A((m == 0 ? 1.0 : 2.0) * (bx ? bx[m] : 1.0)), wm1 = A(2.0 * (bx ? bx[m + 1] : 1.0));
    if (k == 0) {
      // the self-paired outputs 0 and N/2; the (0,0) coefficient is zero
      const C V0 = x[F::out_slot(0)], Vh = x[F::out_slot(N / 2)];
      const A e0 = Ew[0].x, eh = Ew[N / 2].x;
      put(0, m, m == 0 ? A(0.0) : e0 * (V0.x + V0.x) * wm0, e0 * (V0.y + V0.y) * wm1);
      put(N / 2, m, eh * (Vh.x + Vh.x) * wm0, eh * (Vh.y + Vh.y) * wm1);
    } else {
      const int q = N - k;
      const C Vn = x[F::out_slot(k)], Vq = x[F::out_slot(q)];
      const A u = Vn.x + Vq.x, v = Vn.y - Vq.y, w = Vn.y + Vq.y, z = Vn.x - Vq.x;
      const C en = Ew[k], eq = Ew[q];
      put(k, m, (en.x * u + en.y * v) * wm0, (en.x * w - en.y * z) * wm1);
      put(q, m, (eq.x * u - eq.y * v) * wm0, (eq.x * w + eq.y * z) * wm1);
    }
  }
}

}  // namespace cg
