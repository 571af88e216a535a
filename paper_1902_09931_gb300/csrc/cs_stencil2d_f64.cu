// FP64-storage instantiation of the 2D stencil kernels (separate unit for parallel builds).
#include "cs_stencil2d_kernels.cuh"

// the TMA sweeps are instantiated in cs_stencil2d_f64_tma.cu (compiled in parallel)
namespace cs {
namespace s2d {
extern template int dispatch_tma<0, double>(int variant, const CUtensorMap& map, const double* in, double* out, int64_t nx, int64_t ny, int periodic, const Taps<double>& taps, const IxTaps& it, const DDTaps& dt, int* status, int stall_from, cudaStream_t st);
extern template int dispatch_tma<1, double>(int variant, const CUtensorMap& map, const double* in, double* out, int64_t nx, int64_t ny, int periodic, const Taps<double>& taps, const IxTaps& it, const DDTaps& dt, int* status, int stall_from, cudaStream_t st);
extern template int dispatch_tma<2, double>(int variant, const CUtensorMap& map, const double* in, double* out, int64_t nx, int64_t ny, int periodic, const Taps<double>& taps, const IxTaps& it, const DDTaps& dt, int* status, int stall_from, cudaStream_t st);
}  // namespace s2d
}  // namespace cs

namespace cs {
int stencil2d_launch_f64(const Stencil2DConfig* cfg, const void* in, void* out, cudaStream_t s) {
  return s2d::launch_stencil2d_t<double>(cfg, in, out, s);
}
int stencil2d_group_f64(const Stencil2DConfig* const* cfgs, const void* const* ins, void* const* outs,
                        int count, cudaStream_t s) {
  return s2d::launch_group_t<double>(cfgs, ins, outs, count, s);
}
}  // namespace cs
