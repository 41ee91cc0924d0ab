// Size dispatch of the spectral kernels for one element type (included by
// spectral_f32.cu and spectral_f64.cu, which instantiate it).
#pragma once

#include "kernels.h"
#include "spectral.cuh"

#define CG_FOR_EACH_LOG2N(X) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

namespace cg {

template <typename T>
cudaError_t prepare_spectral(int log2Lx, int log2Ly) {
  // allow the largest shared memory any tuning candidate needs
  const int Lx = 1 << log2Lx, Ly = 1 << log2Ly;
  LaunchCfg r = inv_rows_cfg(log2Lx, Ly, sizeof(T), 1), c = inv_cols_cfg(log2Ly, Lx, sizeof(T), 2);
  for (int S = 1; S <= 16 && S <= Ly; S *= 2) {
    const LaunchCfg k = inv_rows_cfg(log2Lx, Ly, sizeof(T), S);
    if (k.smem <= 227 * 1024 && k.smem > r.smem) r = k;
  }
  for (int W = 2; W <= 16 && W <= Lx; W *= 2) {
    const LaunchCfg k = inv_cols_cfg(log2Ly, Lx, sizeof(T), W);
    if (k.smem <= 227 * 1024 && k.smem > c.smem) c = k;
  }
  const LaunchCfg f = fwd_cols_cfg(log2Ly, Lx);
  cudaError_t e = cudaSuccess;
  switch (log2Lx) {
#define CG_CASE(L)                                                                             \
  case L:                                                                                      \
    e = cudaFuncSetAttribute((const void*)inv_rows_kernel<T, L>,                               \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r.smem);        \
    break;
    CG_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  switch (log2Ly) {
#define CG_CASE(L)                                                                             \
  case L:                                                                                      \
    e = cudaFuncSetAttribute((const void*)inv_cols_kernel<T, L>,                               \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);        \
    if (e == cudaSuccess)                                                                      \
      e = cudaFuncSetAttribute((const void*)fwd_cols_kernel<T, L>,                             \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.smem);      \
    break;
    CG_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: return cudaErrorInvalidValue;
  }
  return e;
}

template <typename T>
cudaError_t spectral_max_threads(int log2Lx, int log2Ly, int* rows_max, int* cols_max) {
  // the largest block each inverse pass can launch with (its registers per thread decide)
  cudaFuncAttributes fa;
  cudaError_t e = cudaErrorInvalidValue;
  switch (log2Lx) {
#define CG_CASE(L)                                                       \
  case L:                                                                \
    e = cudaFuncGetAttributes(&fa, (const void*)inv_rows_kernel<T, L>); \
    break;
    CG_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
  if (e != cudaSuccess) return e;
  *rows_max = fa.maxThreadsPerBlock;
  e = cudaErrorInvalidValue;
  switch (log2Ly) {
#define CG_CASE(L)                                                       \
  case L:                                                                \
    e = cudaFuncGetAttributes(&fa, (const void*)inv_cols_kernel<T, L>); \
    break;
    CG_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
  if (e != cudaSuccess) return e;
  *cols_max = fa.maxThreadsPerBlock;
  return cudaSuccess;
}

template <typename T>
void launch_inv_rows(int log2Lx, int Ly, int S, const T* spec, V2<T>* AB, const V2<T>* W,
                     const V2<T>* E, DevState* st, int mode, double tau,
                     cudaGraphConditionalHandle handle, int use_cond, unsigned int max_body,
                     cudaStream_t s) {
  const LaunchCfg c = inv_rows_cfg(log2Lx, Ly, sizeof(T), S);
  switch (log2Lx) {
#define CG_CASE(L)                                                                                \
  case L:                                                                                         \
    launch_pdl(inv_rows_kernel<T, L>, c.grid, c.threads, c.smem, s, spec, AB, W, E, Ly,        \
               c.per_block, st, mode, tau, handle, use_cond, max_body);                          \
    break;
    CG_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
}

template <typename T>
void launch_inv_cols(int log2Ly, int Lx, int Wc, const V2<T>* AB, V2<T>* v0, V2<T>* v1,
                     T* rho_out, const V2<T>* W, const V2<T>* E, DevState* st, int mode,
                     cudaStream_t s) {
  const LaunchCfg c = inv_cols_cfg(log2Ly, Lx, sizeof(T), Wc);
  switch (log2Ly) {
#define CG_CASE(L)                                                                              \
  case L:                                                                                       \
    launch_pdl(inv_cols_kernel<T, L>, c.grid, c.threads, c.smem, s, AB, v0, v1, rho_out, W, E, \
               Lx, c.per_block, st, mode);                                                      \
    break;
    CG_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
}

template <typename T>
void launch_fwd(int log2Lx, int log2Ly, const double* rho, double* R, double* spec64, T* specT,
                const double2* Wx, const double2* Ex, const double2* Wy, const double2* Ey,
                const double* bx, const double* by, cudaStream_t s) {
  const int Lx = 1 << log2Lx;
  launch_fwd_rows(log2Lx, log2Ly, rho, R, Wx, Ex, s);
  const LaunchCfg c = fwd_cols_cfg(log2Ly, Lx);
  switch (log2Ly) {
#define CG_CASE(L)                                                                                 \
  case L:                                                                                          \
    fwd_cols_kernel<T, L><<<c.grid, c.threads, c.smem, s>>>(R, spec64, specT, Wy, Ey, bx, by, Lx, \
                                                            c.per_block);                          \
    break;
    CG_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
}

#define CG_INSTANTIATE_SPECTRAL(T)                                                                 \
  template cudaError_t prepare_spectral<T>(int, int);                                              \
  template cudaError_t spectral_max_threads<T>(int, int, int*, int*);                              \
  template void launch_inv_rows<T>(int, int, int, const T*, V2<T>*, const V2<T>*, const V2<T>*,   \
                                   DevState*, int, double, cudaGraphConditionalHandle, int,        \
                                   unsigned int, cudaStream_t);                                    \
  template void launch_inv_cols<T>(int, int, int, const V2<T>*, V2<T>*, V2<T>*, T*, const V2<T>*, \
                                   const V2<T>*, DevState*, int, cudaStream_t);                    \
  template void launch_fwd<T>(int, int, const double*, double*, double*, T*, const double2*,      \
                              const double2*, const double2*, const double2*, const double*,       \
                              const double*, cudaStream_t);

}  // namespace cg
