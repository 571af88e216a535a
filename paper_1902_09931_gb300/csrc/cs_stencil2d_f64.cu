// FP64-storage instantiation of the 2D stencil kernels (separate unit for parallel builds).
#include "cs_stencil2d_kernels.cuh"

namespace cs {
int stencil2d_launch_f64(const Stencil2DConfig* cfg, const void* in, void* out, cudaStream_t s) {
  return s2d::launch_stencil2d_t<double>(cfg, in, out, s);
}
}  // namespace cs
