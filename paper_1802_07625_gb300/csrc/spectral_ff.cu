// Float-float kernels (size dispatch): pass 2 of the inverse transform on FP32 data (the
// compensated mixed precision) and the forward transform of the mixed precisions.
#include "ff.cuh"
#include "kernels.h"
#include "spectral.cuh"

#define CG_FF_FOR_EACH_LOG2N(X) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

namespace cg {

cudaError_t prepare_spectral_ff(int log2Ly, int Lx, int* cols_max_threads) {
  LaunchCfg c = inv_cols_ff_cfg(log2Ly, Lx, 2);
  for (int W = 2; W <= 16 && W <= Lx; W *= 2) {
    const LaunchCfg k = inv_cols_ff_cfg(log2Ly, Lx, W);
    if (k.smem <= 227 * 1024 && k.smem > c.smem) c = k;
  }
  cudaError_t e = cudaErrorInvalidValue;
  cudaFuncAttributes fa;
  switch (log2Ly) {
#define CG_CASE(L)                                                                                 \
  case L:                                                                                          \
    e = cudaFuncSetAttribute((const void*)inv_cols_kernel<float, L, ff>,                           \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);            \
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)inv_cols_kernel<float, L, ff>); \
    break;
    CG_FF_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
  if (e == cudaSuccess && cols_max_threads) *cols_max_threads = fa.maxThreadsPerBlock;
  return e;
}

void launch_inv_cols_ff(int log2Ly, int Lx, int Wc, const float2* AB, float2* v0, float2* v1, float* rho_out,
                        const void* W, const void* E, DevState* st, int mode, cudaStream_t s) {
  const LaunchCfg c = inv_cols_ff_cfg(log2Ly, Lx, Wc);
  const ff2* Wf = static_cast<const ff2*>(W);
  const ff2* Ef = static_cast<const ff2*>(E);
  switch (log2Ly) {
#define CG_CASE(L)                                                                                  \
  case L:                                                                                           \
    launch_pdl(inv_cols_kernel<float, L, ff>, c.grid, c.threads, c.smem, s, AB, v0, v1, rho_out, Wf, \
               Ef, Lx, c.per_block, st, mode);                                                      \
    break;
    CG_FF_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
}

cudaError_t prepare_forward_ff(int log2Lx, int log2Ly) {
  const LaunchCfg r = fwd_rows_cfg(log2Lx, 1 << log2Ly), c = fwd_cols_cfg(log2Ly, 1 << log2Lx);
  cudaError_t e = cudaErrorInvalidValue;
  switch (log2Lx) {
#define CG_CASE(L)                                                                                  \
  case L:                                                                                           \
    e = cudaFuncSetAttribute((const void*)fwd_rows_kernel<L, ff>,                                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r.smem);             \
    break;
    CG_FF_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
  if (e != cudaSuccess) return e;
  e = cudaErrorInvalidValue;
  switch (log2Ly) {
#define CG_CASE(L)                                                                                  \
  case L:                                                                                           \
    e = cudaFuncSetAttribute((const void*)fwd_cols_kernel<float, L, ff>,                            \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);             \
    break;
    CG_FF_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
  return e;
}

void launch_fwd_ff(int log2Lx, int log2Ly, const double* rho, double* R, double* spec64, float* specT,
                   const void* Wx, const void* Ex, const void* Wy, const void* Ey, const double* bx,
                   const double* by, cudaStream_t s) {
  const int Lx = 1 << log2Lx;
  const LaunchCfg r = fwd_rows_cfg(log2Lx, 1 << log2Ly), c = fwd_cols_cfg(log2Ly, Lx);
  const ff2 *Wxf = static_cast<const ff2*>(Wx), *Exf = static_cast<const ff2*>(Ex);
  const ff2 *Wyf = static_cast<const ff2*>(Wy), *Eyf = static_cast<const ff2*>(Ey);
  switch (log2Lx) {
#define CG_CASE(L)                                                                                  \
  case L:                                                                                           \
    fwd_rows_kernel<L, ff><<<r.grid, r.threads, r.smem, s>>>(rho, R, Wxf, Exf, r.per_block);        \
    break;
    CG_FF_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
  switch (log2Ly) {
#define CG_CASE(L)                                                                                  \
  case L:                                                                                           \
    fwd_cols_kernel<float, L, ff><<<c.grid, c.threads, c.smem, s>>>(R, spec64, specT, Wyf, Eyf, bx, by, \
                                                                    Lx, c.per_block);              \
    break;
    CG_FF_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
}

}  // namespace cg
