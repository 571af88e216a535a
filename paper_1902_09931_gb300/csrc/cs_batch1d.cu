// Batched 1D stencil over a ragged, packed set of lines (Abstract; Sec. 5.4 "batches of 1D
// problems"; the X-direction stencil of Sec. 3 applied to each line on its own).
//
// out[k] = sum_p w[p] * in[line_start + wrap(k - line_start - left + p, line_len)]   (periodic)
//
// The packed buffer is cut into warp segments of 32 lanes x 32 bytes, independent of where
// lines start, so every warp does the same amount of work whatever the length mix.  A
// persistent grid-stride launch walks the segments.  Each lane loads two 16-byte vectors, takes
// its left / right neighbours from the adjacent lanes with warp shuffles (lanes 0 and 31 load
// the few values beyond the segment), and forms its sums uniformly.  A table that maps every
// 64th element to the line containing it (built once at create time) gives the line of the
// segment's first element; lanes 0..3 load that line's start and the next three line
// boundaries, which reach every lane by shuffle, so a lane finds its line with two compares.
// An element is written by the segment walk only when its stencil stays inside its line; the
// first L and last R elements of every periodic line (whose stencils wrap) are then written by
// the same launch, one thread per such element, and those of a non-periodic line are left
// untouched.  Stencils wider than the vector width take a per-element kernel.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>

#include "cs_internal.h"

namespace cs {
namespace {

constexpr int kSegShift = 6;  // table granularity: one entry per 64 packed elements

template <typename T> struct Vec1;
template <> struct Vec1<float> { static constexpr int n = 4; using V = float4; };
template <> struct Vec1<double> { static constexpr int n = 2; using V = double2; };

template <typename T> struct BTaps { T w[2 * CS_MAX_EXTENT + 1]; };

struct LaunchShape { int threads, ctas_per_sm; };
constexpr LaunchShape kShapes[] = {{256, 4}, {256, 8}, {512, 2}, {128, 8}, {512, 1}, {256, 2}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

__global__ void k_build_seg_table(const int64_t* __restrict__ off, int64_t num_lines,
                                  int64_t ntab, int32_t* __restrict__ seg) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= ntab) return;
  const int64_t k = t << kSegShift;
  // largest m in [0, num_lines) with off[m] <= k
  int64_t lo = 0, hi = num_lines - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  seg[t] = static_cast<int32_t>(lo);
}

// Per-element evaluation of elements k0 .. k0 + n - 1 with wrapped loads: lanes beyond a
// segment's fourth line boundary (lines shorter than a segment) and stencils wider than the
// vector width.  m, ls, le: a line at or before the one holding k0, and its bounds.
template <typename T>
__device__ __forceinline__ void elements_general(const T* __restrict__ in, T* __restrict__ out,
                                                 const int64_t* __restrict__ off, int64_t total,
                                                 int periodic, int L, int R, const BTaps<T>& taps,
                                                 int64_t k0, int n, int64_t m, int64_t ls, int64_t le) {
  const int W = L + R + 1;
  for (int e = 0; e < n; ++e) {
    const int64_t k = k0 + e;
    if (k >= total) break;
    while (k >= le) {  // advance to the line holding k (skips empty lines)
      ++m;
      ls = le;
      le = __ldg(off + m + 1);
    }
    const int64_t len = le - ls;
    if (!periodic && (k - ls < L || le - 1 - k < R)) continue;  // boundary cell untouched
    const int rel0 = static_cast<int>(k - ls) - L;  // lines hold < 2^31 elements
    const int ilen = static_cast<int>(len);
    T acc = T(0);
    for (int p = 0; p < W; ++p) {
      int rel = (rel0 + p) % ilen;
      if (rel < 0) rel += ilen;
      acc = fma(taps.w[p], __ldg(in + ls + rel), acc);
    }
    out[k] = acc;
  }
}

// Elements per lane: two 16-byte vectors, so the per-segment work (line boundaries, shuffles,
// classification) is shared by 8 FP32 or 4 FP64 elements.
constexpr int kLaneVecs = 2;
template <typename T> constexpr int lane_elems() { return kLaneVecs * Vec1<T>::n; }

// One warp segment of 32 * E packed elements starting at s: own values v (already loaded),
// neighbours by shuffle (lanes 0 and 31 take the nearest L / R values of the adjacent segments
// from hl / hr, loaded with the segment), the lane's line from the segment's boundaries, and the
// weighted sum.  r holds, on lanes 0..3, the boundary off[m0 + lane] relative to s (clamped;
// total past the last line), m0 the line of s.  Elements whose stencil would cross the end of
// their line are not written here.
template <typename T, int LL, int RR>
__device__ __forceinline__ void segment(const T* __restrict__ in, T* __restrict__ out,
                                        const int64_t* __restrict__ off, int64_t total,
                                        int Lr, int Rr, bool vec_ok,
                                        const BTaps<T>& taps, int64_t s, int64_t m0, int r,
                                        const T (&v)[lane_elems<T>()], const T (&hl)[LL > 0 ? LL : 1],
                                        const T (&hr)[RR > 0 ? RR : 1]) {
  constexpr int V = Vec1<T>::n, E = lane_elems<T>();
  using VT = typename Vec1<T>::V;
  constexpr int L = LL, R = RR, W = LL + RR + 1;
  static_assert(LL >= 0 && RR >= 0 && LL <= E && RR <= E, "compile-time extents within a lane's elements");
  (void)Lr;
  (void)Rr;
  const int lane = threadIdx.x & 31;
  const int64_t k0 = s + lane * E;
  // win[j]: value at k0 - L + j, j < E + L + R (valid where inside the element's line)
  T win[E + L + R];
#pragma unroll
  for (int e = 0; e < E; ++e) win[L + e] = v[e];
#pragma unroll
  for (int e = 0; e < L; ++e) {
    const T u = __shfl_up_sync(0xffffffffu, v[E - L + e], 1);
    win[e] = lane == 0 ? hl[e] : u;
  }
#pragma unroll
  for (int e = 0; e < R; ++e) {
    const T d = __shfl_down_sync(0xffffffffu, v[e], 1);
    win[L + E + e] = lane == 31 ? hr[e] : d;
  }
  const int r0 = __shfl_sync(0xffffffffu, r, 0), r1 = __shfl_sync(0xffffffffu, r, 1);
  const int r2 = __shfl_sync(0xffffffffu, r, 2), r3 = __shfl_sync(0xffffffffu, r, 3);
  if (k0 >= total) return;
  // every lane forms its E sums from the window; an element is written here only when its
  // stencil stays inside its line (the first L and last R elements of a periodic line are
  // written by the line-ends pass, those of a non-periodic line stay untouched)
  T res[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    T acc = T(0);
#pragma unroll
    for (int p = 0; p < W; ++p) acc = fma(taps.w[p], win[e + p], acc);
    res[e] = acc;
  }
  const int o = lane * E, oe = o + E - 1;
  const int c0 = (o >= r1) + (o >= r2), c1 = (oe >= r1) + (oe >= r2);
  const int ls = c0 == 0 ? r0 : (c0 == 1 ? r1 : r2);
  const int le = c0 == 0 ? r1 : (c0 == 1 ? r2 : r3);
  if (c0 == c1 && oe < r3 && k0 + E <= total && o - L >= ls && oe + R < le) {  // the common case
    if (vec_ok) {
#pragma unroll
      for (int q = 0; q < kLaneVecs; ++q) {
        VT y;
        if constexpr (V == 4) { y.x = res[4 * q]; y.y = res[4 * q + 1]; y.z = res[4 * q + 2]; y.w = res[4 * q + 3]; }
        else { y.x = res[2 * q]; y.y = res[2 * q + 1]; }
        *reinterpret_cast<VT*>(out + k0 + q * V) = y;
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) out[k0 + e] = res[e];
    }
    return;
  }
  if (oe < r3) {  // near a line end: each element's line is one of the segment's three
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int oo = o + e;
      const int ce = (oo >= r1) + (oo >= r2);
      const int ls_e = ce == 0 ? r0 : (ce == 1 ? r1 : r2);
      const int le_e = ce == 0 ? r1 : (ce == 1 ? r2 : r3);
      if (k0 + e < total && oo - ls_e >= L && le_e - 1 - oo >= R) out[k0 + e] = res[e];
    }
    return;
  }
  // more lines in this segment than its four boundaries describe (lines shorter than a
  // segment): walk the offsets from the lane's first line
  int64_t m = m0 + c0, lsa = s + ls, lea = s + le;
  for (int e = 0; e < E; ++e) {
    const int64_t k = k0 + e;
    if (k >= total) break;
    while (k >= lea) {  // skips empty lines
      ++m;
      lsa = lea;
      lea = __ldg(off + m + 1);
    }
    if (k - lsa >= L && lea - 1 - k >= R) out[k] = res[e];
  }
}

// The first L and last R elements of every periodic line, whose stencils wrap around the line:
// items t = m * (L + R) + which in [first, n) with the given stride, taps read from memory at
// their wrapped index (lines shorter than the stencil wrap more than once).
template <typename T>
__device__ __forceinline__ void line_ends(const T* __restrict__ in, T* __restrict__ out,
                                          const int64_t* __restrict__ off, int64_t num_lines,
                                          int L, int R, const BTaps<T>& taps, int64_t first,
                                          int64_t stride) {
  const int B = L + R, W = L + R + 1;
  const int64_t n = num_lines * B;
  for (int64_t t = first; t < n; t += stride) {
    const int64_t m = t / B;
    const int which = static_cast<int>(t - m * B);
    const int64_t ls = __ldg(off + m), le = __ldg(off + m + 1);
    const int len = static_cast<int>(le - ls);  // lines hold < 2^31 elements
    int rel;
    if (which < L) {
      rel = which;
      if (rel >= len) continue;
    } else {
      rel = len - R + (which - L);
      if (rel < L || rel < 0) continue;  // a short line's element already taken from the left
    }
    T acc = T(0);
    for (int p = 0; p < W; ++p) {
      int j = rel - L + p;
      j = j < 0 ? j + len : (j >= len ? j - len : j);
      if (j < 0 || j >= len) {
        j %= len;
        if (j < 0) j += len;
      }
      acc = fma(taps.w[p], __ldg(in + ls + j), acc);
    }
    out[ls + rel] = acc;
  }
}

// Each warp takes kG consecutive segments per iteration and issues all their loads first.
constexpr int kG = 2;

template <typename T, int LL, int RR>
__global__ void k_batch1d(const T* __restrict__ in, T* __restrict__ out,
                          const int64_t* __restrict__ off, const int32_t* __restrict__ seg,
                          int64_t total, int64_t num_lines, int periodic, int Lr, int Rr,
                          int vec_ok, BTaps<T> taps) {
  constexpr int V = Vec1<T>::n, E = lane_elems<T>();
  using VT = typename Vec1<T>::V;
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  constexpr int64_t kSeg = 32 * E;
  static_assert(kSeg % (int64_t(1) << kSegShift) == 0, "segments start on line-table entries");
  const int64_t nseg = (total + kSeg - 1) / kSeg;
  constexpr int kClamp = 1 << 30;
  constexpr int HL = LL > 0 ? LL : 1, HR = RR > 0 ? RR : 1;

  for (int64_t s0 = warp_id * kG; s0 < nseg; s0 += nwarps * kG) {  // warp-uniform loop
    T v[kG][E], hl[kG][HL], hr[kG][HR];
    int64_t m0[kG];
    int r[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) m0[g] = s0 + g < nseg ? __ldg(seg + (((s0 + g) * kSeg) >> kSegShift)) : 0;
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      const int64_t k0 = (s0 + g) * kSeg + lane * E;
      if (vec_ok && k0 + E <= total) {
#pragma unroll
        for (int q = 0; q < kLaneVecs; ++q) {
          const VT x = *reinterpret_cast<const VT*>(in + k0 + q * V);
          if constexpr (V == 4) { v[g][4 * q] = x.x; v[g][4 * q + 1] = x.y; v[g][4 * q + 2] = x.z; v[g][4 * q + 3] = x.w; }
          else { v[g][2 * q] = x.x; v[g][2 * q + 1] = x.y; }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) v[g][e] = (k0 + e < total) ? in[k0 + e] : T(0);
      }
      // lane 0: the L values before the segment; lane 31: the R values after it
#pragma unroll
      for (int e = 0; e < HL; ++e) {
        const int64_t k = k0 - LL + e;
        hl[g][e] = (lane == 0 && e < LL && k >= 0) ? __ldg(in + k) : T(0);
      }
#pragma unroll
      for (int e = 0; e < HR; ++e) {
        const int64_t k = k0 + E + e;
        hr[g][e] = (lane == 31 && e < RR && k < total) ? __ldg(in + k) : T(0);
      }
    }
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      const int64_t s = (s0 + g) * kSeg;
      const int64_t b = (lane < 4 && m0[g] + lane <= num_lines) ? __ldg(off + m0[g] + lane) : total;
      const int64_t d = b - s;
      r[g] = static_cast<int>(d < -kClamp ? -kClamp : (d > kClamp ? kClamp : d));
    }
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      if (s0 + g >= nseg) break;  // warp-uniform
      segment<T, LL, RR>(in, out, off, total, Lr, Rr, vec_ok != 0, taps, (s0 + g) * kSeg,
                         m0[g], r[g], v[g], hl[g], hr[g]);
    }
  }
  // then the wrapped line ends (written by nobody else), spread over all threads
  if (periodic && LL + RR > 0)
    line_ends<T>(in, out, off, num_lines, LL, RR, taps,
                 static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x,
                 static_cast<int64_t>(gridDim.x) * blockDim.x);
}

// Any extents up to CS_MAX_EXTENT: every element on its own, lines found through the table.
template <typename T>
__global__ void k_batch1d_generic(const T* __restrict__ in, T* __restrict__ out,
                                  const int64_t* __restrict__ off, const int32_t* __restrict__ seg,
                                  int64_t total, int64_t num_lines, int periodic, int L, int R,
                                  BTaps<T> taps) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total; k += stride) {
    int64_t m = __ldg(seg + (k >> kSegShift));
    int64_t ls = __ldg(off + m), le = __ldg(off + m + 1);
    (void)num_lines;
    elements_general<T>(in, out, off, total, periodic, L, R, taps, k, 1, m, ls, le);
  }
}

template <typename T, int LL, int RR>
int launch_t(const Batch1DConfig* c, const void* vin, void* vout, cudaStream_t st) {
  const T* in = static_cast<const T*>(vin);
  T* out = static_cast<T*>(vout);
  BTaps<T> taps;
  const int W = c->left + c->right + 1;
  for (int i = 0; i < 2 * CS_MAX_EXTENT + 1; ++i)
    taps.w[i] = i < W ? static_cast<T>(c->weights[i]) : T(0);
  const LaunchShape sh = kShapes[c->choice];
  const bool generic = LL < 0;
  auto kern = generic ? k_batch1d_generic<T> : nullptr;
  int resident = 0;  // persistent grid: never more CTAs than can be resident at once
  if constexpr (LL < 0) {
    CS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_batch1d_generic<T>, sh.threads, 0));
  } else {
    CS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_batch1d<T, LL, RR>, sh.threads, 0));
  }
  (void)kern;
  if (resident < 1)
    return set_error(CS_EUNSUPPORTED, "batched 1D launch shape %d x %d does not fit on an SM", sh.threads, sh.ctas_per_sm);
  const int per_sm = std::min(sh.ctas_per_sm, resident);
  if constexpr (LL < 0) {
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((c->total_len + sh.threads - 1) / sh.threads,
                                                                static_cast<int64_t>(num_sms()) * per_sm));
    k_batch1d_generic<T><<<static_cast<unsigned>(grid), sh.threads, 0, st>>>(
        in, out, c->d_offsets, c->d_seg_line, c->total_len, c->num_lines, c->bc == CS_BC_PERIODIC,
        c->left, c->right, taps);
  } else {
    const int vec_ok = (reinterpret_cast<uintptr_t>(in) % 16 == 0) &&
                       (reinterpret_cast<uintptr_t>(out) % 16 == 0);
    const int64_t seg_elems = 32 * lane_elems<T>();
    const int64_t nseg = (c->total_len + seg_elems - 1) / seg_elems;
    const int64_t warps_per_cta = sh.threads / 32;
    int64_t grid = std::min<int64_t>((nseg + warps_per_cta * kG - 1) / (warps_per_cta * kG),
                                     static_cast<int64_t>(num_sms()) * per_sm);
    grid = std::max<int64_t>(grid, 1);
    k_batch1d<T, LL, RR><<<static_cast<unsigned>(grid), sh.threads, 0, st>>>(
        in, out, c->d_offsets, c->d_seg_line, c->total_len, c->num_lines, c->bc == CS_BC_PERIODIC,
        c->left, c->right, vec_ok, taps);
  }
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

// Extents up to 2 on either side (within one vector of both storage types) get a kernel with the
// extents compiled in; wider stencils take the per-element kernel.
template <typename T>
int launch_dispatch(const Batch1DConfig* c, const void* in, void* out, cudaStream_t st) {
  switch (c->left * 3 + c->right) {
#define CS_B1_CASE(A, B) \
  case A * 3 + B: if (c->left == A && c->right == B) return launch_t<T, A, B>(c, in, out, st); break;
    CS_B1_CASE(0, 0) CS_B1_CASE(0, 1) CS_B1_CASE(0, 2) CS_B1_CASE(1, 0) CS_B1_CASE(1, 1)
    CS_B1_CASE(1, 2) CS_B1_CASE(2, 0) CS_B1_CASE(2, 1) CS_B1_CASE(2, 2)
#undef CS_B1_CASE
    default: break;
  }
  return launch_t<T, -1, -1>(c, in, out, st);
}

}  // namespace

int batch1d_prepare(Batch1DConfig* c, cudaStream_t st) {
  c->d_seg_line = nullptr;
  c->num_table = 0;
  c->choice = 1;
  if (c->total_len == 0) return CS_OK;
  c->num_table = ((c->total_len - 1) >> kSegShift) + 1;
  CS_CUDA_TRY(cudaMalloc(&c->d_seg_line, c->num_table * sizeof(int32_t)));
  const int threads = 256;
  k_build_seg_table<<<static_cast<unsigned>((c->num_table + threads - 1) / threads), threads, 0, st>>>(
      c->d_offsets, c->num_lines, c->num_table, c->d_seg_line);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  int choice;
  if (tune_lookup(batch1d_shape_key(c), &choice) && choice >= 0 && choice < kNumShapes)
    c->choice = choice;
  return CS_OK;
}

void batch1d_release(Batch1DConfig* c) {
  if (c->d_seg_line) cudaFree(c->d_seg_line);
  c->d_seg_line = nullptr;
}

int batch1d_num_choices() { return kNumShapes; }

std::string batch1d_shape_key(const Batch1DConfig* c) {
  char buf[160];
  const double mean = c->num_lines > 0 ? static_cast<double>(c->total_len) / c->num_lines : 0.0;
  const int mean_class = mean < 128 ? 0 : mean < 1024 ? 1 : 2;
  const int size_class = c->total_len <= (1 << 20) ? 0 : c->total_len <= (1 << 24) ? 1 : 2;
  snprintf(buf, sizeof buf, "batch1d|%s|e%d.%d_bc%d_m%d_s%d|sm%d", c->dtype == CS_F32 ? "f32" : "f64",
           c->left, c->right, c->bc, mean_class, size_class, num_sms());
  return buf;
}

int batch1d_launch(const Batch1DConfig* c, const void* in, void* out, cudaStream_t st) {
  if (c->total_len == 0) return CS_OK;
  return c->dtype == CS_F32 ? launch_dispatch<float>(c, in, out, st)
                            : launch_dispatch<double>(c, in, out, st);
}

}  // namespace cs

// ---- allocation-free entry point --------------------------------------------------------------
// Some callers cannot let a library call cudaMalloc: code that runs under a fixed device-memory
// budget or an arena owned by another runtime, latency-critical loops where an allocation (and
// its implicit synchronisation) is not acceptable, or plain C callers that only hand over
// buffers they already own.  cs_batch1d_compute_noalloc serves them: it runs the batched 1D
// sweep with the line-lookup table kept in the file-scope array below instead of in a plan's
// cudaMalloc'ed workspace.  The array is created when the library is loaded and every GPU that
// loads the library holds it (4 MiB + 256 B) until the process exits.

namespace cs {
namespace {

constexpr int64_t kNoAllocTableEntries = int64_t(1) << 20;                     // line-table entries
constexpr int64_t kNoAllocMaxLen = kNoAllocTableEntries << kSegShift;         // 2^26 elements
constexpr int64_t kNoAllocStatusSlot = kNoAllocTableEntries;                  // validation flag

// Line table (one entry per 64 packed elements) followed by a 64-entry tail whose first word is
// the offsets-validation flag.  Shared by every call in the process.
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocTableEntries + 64];

// Device address of g_noalloc_scratch, looked up once per device (the host-side name is only a
// stand-in for the symbol, not a device pointer).
std::atomic<int32_t*> g_noalloc_addr[64];

__global__ void k_check_offsets(const int64_t* __restrict__ off, int64_t num_lines, int64_t total,
                                int32_t* __restrict__ status) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t m = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; m < num_lines; m += stride)
    if (off[m] > off[m + 1]) atomicOr(status, 1);
  if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[num_lines] != total)) atomicOr(status, 2);
}

int noalloc_scratch(int32_t** out) {
  int dev = 0;
  CS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(CS_EUNSUPPORTED, "device index %d out of range", dev);
  int32_t* p = g_noalloc_addr[dev].load();
  if (!p) {
    void* addr = nullptr;
    CS_CUDA_TRY(cudaGetSymbolAddress(&addr, g_noalloc_scratch));
    p = static_cast<int32_t*>(addr);
    g_noalloc_addr[dev].store(p);
  }
  *out = p;
  return CS_OK;
}

}  // namespace

}  // namespace cs

extern "C" int cs_batch1d_compute_noalloc(const cs_stencil_desc* d, int64_t num_lines,
                                          const int64_t* d_offsets, int64_t total_len,
                                          const void* d_in, void* d_out, void* stream) {
  using namespace cs;
  if (!d) return set_error(CS_EINVAL, "null stencil description");
  if (d->dtype != CS_F64 && d->dtype != CS_F32) return set_error(CS_EINVAL, "dtype must be CS_F64 or CS_F32");
  if (d->bc != CS_BC_PERIODIC && d->bc != CS_BC_NONPERIODIC) return set_error(CS_EINVAL, "bc must be periodic or non-periodic");
  if (d->dir != CS_DIR_X || d->top != 0 || d->bottom != 0 || d->fn != CS_FN_NONE || !d->weights)
    return set_error(CS_EINVAL, "batched 1D lines take a weighted X stencil");
  if (d->left < 0 || d->right < 0 || d->left > CS_MAX_EXTENT || d->right > CS_MAX_EXTENT)
    return set_error(CS_EINVAL, "stencil extents must be in [0, %d]", CS_MAX_EXTENT);
  if (num_lines < 0 || total_len < 0 || num_lines > 0x7fffffff)
    return set_error(CS_EINVAL, "num_lines, total_len out of range");
  if (total_len > kNoAllocMaxLen)
    return set_error(CS_EINVAL, "cs_batch1d_compute_noalloc: total_len %lld exceeds the fixed maximum %lld (use a plan)",
                     (long long)total_len, (long long)kNoAllocMaxLen);
  if (total_len > 0 && num_lines == 0) return set_error(CS_EINVAL, "elements without lines");
  if (!d_offsets) return set_error(CS_EINVAL, "null offsets");
  if (total_len == 0) return CS_OK;
  const size_t eb = d->dtype == CS_F32 ? 4 : 8;
  if (!d_in || !d_out) return set_error(CS_EINVAL, "null device buffer");
  if (reinterpret_cast<uintptr_t>(d_in) % eb || reinterpret_cast<uintptr_t>(d_out) % eb)
    return set_error(CS_EINVAL, "buffers must be aligned to the element size");
  {
    const char* a = static_cast<const char*>(d_in);
    const char* b = static_cast<const char*>(d_out);
    const size_t bytes = static_cast<size_t>(total_len) * eb;
    if (a < b + bytes && b < a + bytes) return set_error(CS_EALIAS, "input and output buffers overlap");
  }
  int32_t* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != CS_OK) return rc;
  int32_t* status = scratch + kNoAllocStatusSlot;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear the flag, then validate the offsets
  CS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  const int64_t check_blocks = std::min<int64_t>((num_lines + 255) / 256, 1024);
  k_check_offsets<<<static_cast<unsigned>(std::max<int64_t>(check_blocks, 1)), 256, 0, st>>>(d_offsets, num_lines, total_len, status);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  int32_t h_status = 0;
  CS_CUDA_TRY(cudaMemcpyAsync(&h_status, status, sizeof h_status, cudaMemcpyDeviceToHost, st));
  CS_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_status != 0)
    return set_error(CS_EINVAL, "offsets must start at 0, end at total_len and be non-decreasing");
  Batch1DConfig c;
  memset(&c, 0, sizeof c);
  c.num_lines = num_lines;
  c.total_len = total_len;
  c.bc = d->bc;
  c.dtype = d->dtype;
  c.left = d->left;
  c.right = d->right;
  for (int i = 0; i < d->left + d->right + 1; ++i) c.weights[i] = d->weights[i];
  c.d_offsets = d_offsets;
  c.d_seg_line = scratch;
  c.num_table = ((total_len - 1) >> kSegShift) + 1;
  c.choice = 1;
  int choice;
  if (tune_lookup(batch1d_shape_key(&c), &choice) && choice >= 0 && choice < kNumShapes) c.choice = choice;
  const int threads = 256;
  k_build_seg_table<<<static_cast<unsigned>((c.num_table + threads - 1) / threads), threads, 0, st>>>(
      d_offsets, num_lines, c.num_table, scratch);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return batch1d_launch(&c, d_in, d_out, st);
}
