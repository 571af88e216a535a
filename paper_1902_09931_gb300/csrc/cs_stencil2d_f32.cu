// FP32-storage instantiation of the 2D stencil kernels (separate unit for parallel builds).
#include "cs_stencil2d_kernels.cuh"

// the TMA sweeps are instantiated in cs_stencil2d_f32_tma.cu (compiled in parallel)
namespace cs {
namespace s2d {
extern template int dispatch_tma<0, float>(int variant, const CUtensorMap& map, const float* in, float* out, int64_t nx, int64_t ny, int periodic, const Taps<float>& taps, const IxTaps& it, const DDTaps& dt, int* status, int stall_from, cudaStream_t st);
}  // namespace s2d
}  // namespace cs

namespace cs {
int stencil2d_launch_f32(const Stencil2DConfig* cfg, const void* in, void* out, cudaStream_t s) {
  return s2d::launch_stencil2d_t<float>(cfg, in, out, s);
}
int stencil2d_group_f32(const Stencil2DConfig* const* cfgs, const void* const* ins, void* const* outs,
                        int count, cudaStream_t s) {
  return s2d::launch_group_t<float>(cfgs, ins, outs, count, s);
}
}  // namespace cs
