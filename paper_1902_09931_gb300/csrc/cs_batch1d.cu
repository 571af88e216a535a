// Batched 1D stencil over a ragged, packed set of lines (Abstract; Sec. 5.4 "batches of 1D
// problems"; the X-direction stencil of Sec. 3 applied to each line on its own).
//
// out[k] = sum_p w[p] * in[line_start + wrap(k - line_start - left + p, line_len)]   (periodic)
//
// The packed buffer is cut into warp segments of 32 lanes x 16 bytes, independent of where
// lines start, so every warp does the same amount of work whatever the length mix.  A
// persistent grid-stride launch walks the segments.  Each lane loads its 16-byte vector, takes
// its left / right neighbours from the adjacent lanes with warp shuffles (lanes 0 and 31 load
// the two ends), and finds its line through a table that maps every 64th element to the line
// containing it (built once at create time), so the lookup is at most a short binary search.
// Lanes whose stencil crosses a line end take a slow path with per-element wrapped loads.
#include <algorithm>
#include <cstdio>

#include "cs_internal.h"

namespace cs {
namespace {

constexpr int kSegShift = 6;  // table granularity: one entry per 64 packed elements

template <typename T> struct Vec1;
template <> struct Vec1<float> { static constexpr int n = 4; using V = float4; };
template <> struct Vec1<double> { static constexpr int n = 2; using V = double2; };

template <typename T> struct BTaps { T w[2 * CS_MAX_EXTENT + 1]; };

struct LaunchShape { int threads, ctas_per_sm; };
constexpr LaunchShape kShapes[] = {{256, 4}, {256, 8}, {512, 4}, {128, 16}, {1024, 2}};
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

__device__ __forceinline__ int64_t find_line(int64_t k, const int64_t* __restrict__ off,
                                             const int32_t* __restrict__ seg, int64_t ntab,
                                             int64_t num_lines) {
  const int64_t t = k >> kSegShift;
  int64_t lo = seg[t];
  int64_t hi = (t + 1 < ntab) ? seg[t + 1] : num_lines - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T, int LL, int RR>
__global__ void k_batch1d(const T* __restrict__ in, T* __restrict__ out,
                          const int64_t* __restrict__ off, const int32_t* __restrict__ seg,
                          int64_t ntab, int64_t total, int64_t num_lines, int periodic,
                          int Lr, int Rr, int vec_ok, BTaps<T> taps) {
  constexpr int V = Vec1<T>::n;
  using VT = typename Vec1<T>::V;
  const int L = LL >= 0 ? LL : Lr;
  const int R = RR >= 0 ? RR : Rr;
  const int W = L + R + 1;
  const bool shuffle_ok = L <= V && R <= V;
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  constexpr int64_t kSeg = 32 * V;
  const int64_t nseg = (total + kSeg - 1) / kSeg;

  for (int64_t s = warp_id; s < nseg; s += nwarps) {  // warp-uniform loop
    const int64_t k0 = s * kSeg + lane * V;
    T v[V];
    if (vec_ok && k0 + V <= total) {
      const VT x = *reinterpret_cast<const VT*>(in + k0);
      if constexpr (V == 4) { v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w; }
      else { v[0] = x.x; v[1] = x.y; }
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) v[e] = (k0 + e < total) ? in[k0 + e] : T(0);
    }
    // window[0 .. 3V): values at k0 - V .. k0 + 2V - 1 (valid where inside the same line)
    T win[3 * V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      win[e] = __shfl_up_sync(0xffffffffu, v[e], 1);
      win[V + e] = v[e];
      win[2 * V + e] = __shfl_down_sync(0xffffffffu, v[e], 1);
    }
    if (k0 >= total) continue;
    if (lane == 0) {
#pragma unroll
      for (int e = 0; e < V; ++e) win[e] = (k0 - V + e >= 0) ? in[k0 - V + e] : T(0);
    }
    if (lane == 31) {
#pragma unroll
      for (int e = 0; e < V; ++e) win[2 * V + e] = (k0 + V + e < total) ? in[k0 + V + e] : T(0);
    }
    int64_t m = find_line(k0, off, seg, ntab, num_lines);
    int64_t ls = __ldg(off + m), le = __ldg(off + m + 1);
    const bool fast = shuffle_ok && k0 + V <= total && k0 - L >= ls && k0 + V - 1 + R < le;
    if (fast) {
      T res[V];
#pragma unroll
      for (int e = 0; e < V; ++e) {
        T acc = T(0);
        if constexpr (LL >= 0 && RR >= 0) {
#pragma unroll
          for (int p = 0; p < LL + RR + 1; ++p) acc = fma(taps.w[p], win[V + e - LL + p], acc);
        } else {
          for (int p = 0; p < W; ++p) acc = fma(taps.w[p], win[V + e - L + p], acc);
        }
        res[e] = acc;
      }
      if (vec_ok) {
        VT y;
        if constexpr (V == 4) { y.x = res[0]; y.y = res[1]; y.z = res[2]; y.w = res[3]; }
        else { y.x = res[0]; y.y = res[1]; }
        *reinterpret_cast<VT*>(out + k0) = y;
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e) out[k0 + e] = res[e];
      }
    } else {
      for (int e = 0; e < V; ++e) {
        const int64_t k = k0 + e;
        if (k >= total) break;
        while (k >= le) {  // advance to the line holding k (skips empty lines)
          ++m;
          ls = le;
          le = __ldg(off + m + 1);
        }
        const int64_t len = le - ls;
        if (!periodic && (k - ls < L || le - 1 - k < R)) continue;  // boundary cell untouched
        T acc = T(0);
        for (int p = 0; p < W; ++p) {
          int64_t rel = k - ls - L + p;
          if (periodic) {
            rel %= len;
            if (rel < 0) rel += len;
          }
          acc = fma(taps.w[p], __ldg(in + ls + rel), acc);
        }
        out[k] = acc;
      }
    }
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
  const int vec_ok = (reinterpret_cast<uintptr_t>(in) % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(out) % 16 == 0);
  const LaunchShape sh = kShapes[c->choice];
  const int64_t seg_elems = 32 * Vec1<T>::n;
  const int64_t nseg = (c->total_len + seg_elems - 1) / seg_elems;
  const int64_t warps_per_cta = sh.threads / 32;
  int64_t grid = std::min<int64_t>((nseg + warps_per_cta - 1) / warps_per_cta,
                                   static_cast<int64_t>(num_sms()) * sh.ctas_per_sm);
  grid = std::max<int64_t>(grid, 1);
  k_batch1d<T, LL, RR><<<static_cast<unsigned>(grid), sh.threads, 0, st>>>(
      in, out, c->d_offsets, c->d_seg_line, c->num_table, c->total_len, c->num_lines,
      c->bc == CS_BC_PERIODIC, c->left, c->right, vec_ok, taps);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

template <typename T>
int launch_dispatch(const Batch1DConfig* c, const void* in, void* out, cudaStream_t st) {
  if (c->left == 2 && c->right == 2) return launch_t<T, 2, 2>(c, in, out, st);
  if (c->left == 1 && c->right == 1) return launch_t<T, 1, 1>(c, in, out, st);
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
