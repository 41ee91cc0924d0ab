// Instantiation and launch of the persistent (cooperative) integration kernel.
#include "kernels.h"
#include "persist.cuh"

namespace cg {

template <typename T>
cudaError_t prepare_integrate(size_t smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute((const void*)integrate_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)integrate_kernel<T>,
                                                       kIntegrateThreads, smem);
}

template <typename T>
cudaError_t launch_integrate(const IntegrateArgs<T>& a, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {const_cast<IntegrateArgs<T>*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)integrate_kernel<T>, dim3(grid), dim3(kIntegrateThreads),
                                     args, smem, s);
}

template cudaError_t prepare_integrate<float>(size_t, int*);
template cudaError_t prepare_integrate<double>(size_t, int*);
template cudaError_t launch_integrate<float>(const IntegrateArgs<float>&, int, size_t, cudaStream_t);
template cudaError_t launch_integrate<double>(const IntegrateArgs<double>&, int, size_t, cudaStream_t);

}  // namespace cg
