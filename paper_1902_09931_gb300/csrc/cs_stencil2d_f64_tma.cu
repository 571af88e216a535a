// FP64-storage instantiations of the TMA-pipelined stencil sweep (own unit for parallel builds).
#include "cs_stencil2d_kernels.cuh"

namespace cs {
namespace s2d {
template int dispatch_tma<0, double>(int variant, const CUtensorMap& map, const double* in, double* out, int64_t nx, int64_t ny, int periodic, const Taps<double>& taps, const IxTaps& it, const DDTaps& dt, int* status, int stall_from, cudaStream_t st);
template int dispatch_tma<1, double>(int variant, const CUtensorMap& map, const double* in, double* out, int64_t nx, int64_t ny, int periodic, const Taps<double>& taps, const IxTaps& it, const DDTaps& dt, int* status, int stall_from, cudaStream_t st);
template int dispatch_tma<2, double>(int variant, const CUtensorMap& map, const double* in, double* out, int64_t nx, int64_t ny, int periodic, const Taps<double>& taps, const IxTaps& it, const DDTaps& dt, int* status, int stall_from, cudaStream_t st);
}  // namespace s2d
}  // namespace cs
