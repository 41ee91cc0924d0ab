// FP32 instantiation of the spectral kernels (mixed-precision path).
#include "spectral_impl.cuh"

namespace cg {
CG_INSTANTIATE_SPECTRAL(float)
}  // namespace cg
