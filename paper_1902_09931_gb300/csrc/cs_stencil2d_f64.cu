// FP64-storage instantiation of the 2D stencil kernels (separate unit for parallel builds).
#include "cs_stencil2d_kernels.cuh"

namespace cs {
int stencil2d_launch_f64(const Stencil2DConfig* cfg, const void* in, void* out, cudaStream_t s) {
  return s2d::launch_stencil2d_t<double>(cfg, in, out, s);
}
int stencil2d_group_f64(const Stencil2DConfig* const* cfgs, const void* const* ins, void* const* outs,
                        int count, cudaStream_t s) {
  return s2d::launch_group_t<double>(cfgs, ins, outs, count, s);
}
}  // namespace cs
