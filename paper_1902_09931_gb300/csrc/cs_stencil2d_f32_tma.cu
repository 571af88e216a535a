// FP32-storage instantiations of the TMA-pipelined stencil sweep (own unit for parallel builds).
#include "cs_stencil2d_kernels.cuh"

namespace cs {
namespace s2d {
template int dispatch_tma<0, float>(int variant, const CUtensorMap& map, const float* in, float* out, int64_t nx, int64_t ny, int periodic, const Taps<float>& taps, const IxTaps& it, const DDTaps& dt, int* status, int stall_from, cudaStream_t st);
}  // namespace s2d
}  // namespace cs
