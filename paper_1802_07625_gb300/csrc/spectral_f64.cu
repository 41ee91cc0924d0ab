// FP64 instantiation of the spectral kernels, and the FP64 forward row transform
// shared by both precisions.
#include "spectral_impl.cuh"

namespace cg {
CG_INSTANTIATE_SPECTRAL(double)

cudaError_t prepare_forward(int log2Lx, int log2Ly) {
  const LaunchCfg r = fwd_rows_cfg(log2Lx, 1 << log2Ly);
  switch (log2Lx) {
#define CG_CASE(L)                                                                    \
  case L:                                                                             \
    return cudaFuncSetAttribute((const void*)fwd_rows_kernel<L>,                      \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r.smem);
    CG_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: return cudaErrorInvalidValue;
  }
}

void launch_fwd_rows(int log2Lx, int log2Ly, const double* rho, double* R, const double2* Wx,
                     const double2* Ex, cudaStream_t s) {
  const LaunchCfg r = fwd_rows_cfg(log2Lx, 1 << log2Ly);
  switch (log2Lx) {
#define CG_CASE(L)                                                                      \
  case L:                                                                               \
    fwd_rows_kernel<L><<<r.grid, r.threads, r.smem, s>>>(rho, R, Wx, Ex, r.per_block);  \
    break;
    CG_FOR_EACH_LOG2N(CG_CASE)
#undef CG_CASE
    default: break;
  }
}
}  // namespace cg
