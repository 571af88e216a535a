// 2D stencil sweep kernels (Sec. 2-4 of arXiv:1902.09931), templated on the storage type.
//
// out[j][i] = sum_{q,p} w[q][p] * in[j - top + q][i - left + p]      (Sec. 3, Sec. 5.2 ordering)
//
// Each CTA (256 threads) owns a TX x TY output tile (TX = 128 floats or 64 doubles: one
// 512-byte row segment).  Its input tile plus halo is staged in shared memory with cp.async:
// 16-byte copies for every aligned chunk inside the grid, element copies with the periodic
// wrap (any number of wraps) resolved in the loader for chunks that cross an edge, zero fill
// for non-periodic out-of-grid cells (never read by a written output).  Each thread then owns
// one column of the tile and walks down its rows with a register sliding window of
// (top+bottom+1) x (left+right+1) values, loading one new stencil row from shared memory per
// output row.  Warps write 32 consecutive outputs per row (coalesced).
//
// Specialised kernels fix the extents and the non-zero tap mask at compile time (taps with a
// zero weight are skipped, weights live in the kernel-parameter constant bank); the generic
// kernel takes any extents up to CS_MAX_EXTENT at run time.
#pragma once

#include <stdint.h>

#include "cs_internal.h"

namespace cs {
namespace s2d {

constexpr int kThreads = 256;

template <typename T> struct Vec;
template <> struct Vec<float> { static constexpr int n = 4; };
template <> struct Vec<double> { static constexpr int n = 2; };

template <typename T> constexpr int tile_x() { return 32 * Vec<T>::n; }  // 128 f32 / 64 f64

struct SpecDesc {
  int L, R, T, B;
  uint32_t mask;  // bit q*(L+R+1)+p set = tap (q, p) has a non-zero weight
  int xform;      // 1: stage u^3 - u instead of u (Laplacian of the cubic term, Sec. 5.2)
  int epi;        // 1: add u^3 - u of the centre value to the weighted sum
};

constexpr uint32_t kMask13 = (1u << 2) | (1u << 6) | (1u << 7) | (1u << 8) | (0x1Fu << 10) |
                             (1u << 16) | (1u << 17) | (1u << 18) | (1u << 22);

// Specialisation table (index = Stencil2DConfig::variant).
constexpr SpecDesc kSpecs[] = {
    {1, 1, 1, 1, 0x1FFu, 0, 0},      // 0  3x3 box (9-point Laplacian)
    {1, 1, 1, 1, 0x0BAu, 0, 0},      // 1  5-point cross
    {2, 2, 2, 2, 0x1FFFFFFu, 0, 0},  // 2  5x5 box
    {2, 2, 2, 2, kMask13, 0, 0},     // 3  13-point biharmonic footprint
    {1, 1, 0, 0, 0x7u, 0, 0},        // 4  x, radius 1
    {2, 2, 0, 0, 0x1Fu, 0, 0},       // 5  x, radius 2
    {2, 2, 0, 0, 0x1Bu, 0, 0},       // 6  x, radius 2, zero centre (first derivative)
    {4, 4, 0, 0, 0x1FFu, 0, 0},      // 7  x, radius 4 (8th-order example, Sec. 4.1)
    {0, 0, 1, 1, 0x7u, 0, 0},        // 8  y, radius 1
    {0, 0, 2, 2, 0x1Fu, 0, 0},       // 9  y, radius 2
    {0, 0, 2, 2, 0x1Bu, 0, 0},       // 10 y, radius 2, zero centre
    {0, 0, 4, 4, 0x1FFu, 0, 0},      // 11 y, radius 4
    {1, 1, 1, 1, 0x0BAu, 1, 0},      // 12 Laplacian of u^3 - u            (CS_FN_CH_NONLIN_LAP)
    {1, 1, 1, 1, 0x0BAu, 0, 1},      // 13 u^3 - u + weighted cross          (CS_FN_CUBIC_MINUS_LAP)
};
constexpr int kNumSpecs = sizeof(kSpecs) / sizeof(kSpecs[0]);

template <typename T> struct Taps { T w[32]; };

__device__ __forceinline__ int64_t wrap_idx(int64_t k, int64_t n) {
  int64_t r = k % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename T> __device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename T> __device__ __forceinline__ T cubic_minus(T u) { return u * u * u - u; }

// Stages rows [y0 - top, y0 + TY + bottom) x columns [x0 - LA, x0 + TX + RA) into s
// (pitch = cols).  LA, RA are left/right rounded up to the vector width so every chunk is
// 16-byte aligned in both memories.
template <typename T>
__device__ __forceinline__ void load_tile(T* s, const T* __restrict__ in, int64_t nx, int64_t ny,
                                          bool periodic, bool vec_ok, int64_t x0, int64_t y0,
                                          int top, int LA, int cols, int rows) {
  constexpr int V = Vec<T>::n;
  const int nch = cols / V;
  const int total = rows * nch;
  for (int idx = threadIdx.x; idx < total; idx += kThreads) {
    const int r = idx / nch;
    const int ch = idx - r * nch;
    T* dst = s + r * cols + ch * V;
    int64_t gy = y0 - top + r;
    if (gy < 0 || gy >= ny) {
      if (!periodic) {
#pragma unroll
        for (int e = 0; e < V; ++e) dst[e] = T(0);
        continue;
      }
      gy = wrap_idx(gy, ny);
    }
    const T* row = in + gy * nx;
    const int64_t gx0 = x0 - LA + static_cast<int64_t>(ch) * V;
    if (vec_ok && gx0 >= 0 && gx0 + V <= nx) {
      cp_async16(dst, row + gx0);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) {
        int64_t gx = gx0 + e;
        if (gx < 0 || gx >= nx) {
          if (!periodic) {
            dst[e] = T(0);
            continue;
          }
          gx = wrap_idx(gx, nx);
        }
        cp_async_elem(dst + e, row + gx);
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void xform_tile(T* s, int n) {
  for (int i = threadIdx.x; i < n; i += kThreads) s[i] = cubic_minus(s[i]);
  __syncthreads();
}

template <typename T, int TY, int SPEC>
__global__ void __launch_bounds__(kThreads)
    k_stencil2d_spec(const T* __restrict__ in, T* __restrict__ out, int64_t nx, int64_t ny,
                     int periodic, int vec_ok, Taps<T> taps) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int L = sd.L, R = sd.R, TT = sd.T, BB = sd.B;
  constexpr int V = Vec<T>::n;
  constexpr int TX = tile_x<T>();
  constexpr int LA = (L + V - 1) / V * V, RA = (R + V - 1) / V * V;
  constexpr int COLS = LA + TX + RA, ROWS = TY + TT + BB;
  constexpr int W = L + R + 1, H = TT + BB + 1;
  constexpr int WX = TX / 32, WY = 8 / WX, RW = TY / WY;
  static_assert(W * H <= 32, "tap table too small");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);

  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * TX;
  const int64_t y0 = static_cast<int64_t>(blockIdx.y) * TY;
  load_tile<T>(s, in, nx, ny, periodic != 0, vec_ok != 0, x0, y0, TT, LA, COLS, ROWS);
  if constexpr (sd.xform) xform_tile<T>(s, ROWS * COLS);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = (warp % WX) * 32 + lane;
  const int r0 = (warp / WX) * RW;
  const int64_t gx = x0 + c;
  const bool col_ok = gx < nx && (periodic || (gx >= L && gx < nx - R));
  const T* sc = s + LA + c - L;

  T win[H][W];
#pragma unroll
  for (int q = 0; q < H - 1; ++q)
#pragma unroll
    for (int p = 0; p < W; ++p) win[q + 1][p] = sc[(r0 + q) * COLS + p];

#pragma unroll
  for (int k = 0; k < RW; ++k) {
#pragma unroll
    for (int q = 0; q < H - 1; ++q)
#pragma unroll
      for (int p = 0; p < W; ++p) win[q][p] = win[q + 1][p];
#pragma unroll
    for (int p = 0; p < W; ++p) win[H - 1][p] = sc[(r0 + k + H - 1) * COLS + p];
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < H; ++q)
#pragma unroll
      for (int p = 0; p < W; ++p)
        if ((sd.mask >> (q * W + p)) & 1u) acc = fma(taps.w[q * W + p], win[q][p], acc);
    if constexpr (sd.epi) acc = cubic_minus(win[TT][L]) + acc;
    const int64_t gy = y0 + r0 + k;
    if (col_ok && gy < ny && (periodic || (gy >= TT && gy < ny - BB))) out[gy * nx + gx] = acc;
  }
}

// Any extents up to CS_MAX_EXTENT; weights staged in shared memory after the tile.
template <typename T, int TY>
__global__ void __launch_bounds__(kThreads)
    k_stencil2d_generic(const T* __restrict__ in, T* __restrict__ out, int64_t nx, int64_t ny,
                        int periodic, int vec_ok, int L, int R, int TT, int BB,
                        const T* __restrict__ wts, int xform, int epi) {
  constexpr int V = Vec<T>::n;
  constexpr int TX = tile_x<T>();
  constexpr int WX = TX / 32, WY = 8 / WX, RW = TY / WY;
  const int LA = (L + V - 1) / V * V, RA = (R + V - 1) / V * V;
  const int COLS = LA + TX + RA, ROWS = TY + TT + BB;
  const int W = L + R + 1, H = TT + BB + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* ws = s + ROWS * COLS;
  for (int i = threadIdx.x; i < W * H; i += kThreads) ws[i] = wts[i];

  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * TX;
  const int64_t y0 = static_cast<int64_t>(blockIdx.y) * TY;
  load_tile<T>(s, in, nx, ny, periodic != 0, vec_ok != 0, x0, y0, TT, LA, COLS, ROWS);
  if (xform) xform_tile<T>(s, ROWS * COLS);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = (warp % WX) * 32 + lane;
  const int r0 = (warp / WX) * RW;
  const int64_t gx = x0 + c;
  const bool col_ok = gx < nx && (periodic || (gx >= L && gx < nx - R));
  const T* sc = s + LA + c - L;
  for (int k = 0; k < RW; ++k) {
    const int64_t gy = y0 + r0 + k;
    if (!(col_ok && gy < ny && (periodic || (gy >= TT && gy < ny - BB)))) continue;
    T acc = T(0);
    for (int q = 0; q < H; ++q) {
      const T* srow = sc + (r0 + k + q) * COLS;
      for (int p = 0; p < W; ++p) acc = fma(ws[q * W + p], srow[p], acc);
    }
    if (epi) acc = cubic_minus(sc[(r0 + k + TT) * COLS + L]) + acc;
    out[gy * nx + gx] = acc;
  }
}

template <typename T>
inline size_t tile_smem_bytes(int L, int R, int TT, int BB, int TY, bool generic) {
  constexpr int V = Vec<T>::n;
  const int LA = (L + V - 1) / V * V, RA = (R + V - 1) / V * V;
  size_t b = sizeof(T) * static_cast<size_t>(TY + TT + BB) * (LA + tile_x<T>() + RA);
  if (generic) b += sizeof(T) * static_cast<size_t>((L + R + 1) * (TT + BB + 1));
  return b;
}

template <typename T, int TY, int SPEC>
int launch_spec(const T* in, T* out, int64_t nx, int64_t ny, int periodic, int vec_ok,
                const Taps<T>& taps, cudaStream_t st) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  const size_t smem = tile_smem_bytes<T>(sd.L, sd.R, sd.T, sd.B, TY, false);
  auto kern = k_stencil2d_spec<T, TY, SPEC>;
  static bool attr_set = false;  // per instantiation; set before first launch
  if (!attr_set) {
    CS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem)));
    attr_set = true;
  }
  dim3 grid(static_cast<unsigned>((nx + tile_x<T>() - 1) / tile_x<T>()),
            static_cast<unsigned>((ny + TY - 1) / TY));
  kern<<<grid, kThreads, smem, st>>>(in, out, nx, ny, periodic, vec_ok, taps);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

template <typename T, int TY>
int launch_generic(const T* in, T* out, const Stencil2DConfig* cfg, const T* d_w, int periodic,
                   int vec_ok, int xform, int epi, cudaStream_t st) {
  const size_t smem = tile_smem_bytes<T>(cfg->left, cfg->right, cfg->top, cfg->bottom, TY, true);
  auto kern = k_stencil2d_generic<T, TY>;
  static bool attr_set = false;
  if (!attr_set) {
    // largest tile the generic kernel can be asked for
    const size_t maxb = tile_smem_bytes<T>(CS_MAX_EXTENT, CS_MAX_EXTENT, CS_MAX_EXTENT,
                                           CS_MAX_EXTENT, TY, true);
    CS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(maxb)));
    attr_set = true;
  }
  dim3 grid(static_cast<unsigned>((cfg->nx + tile_x<T>() - 1) / tile_x<T>()),
            static_cast<unsigned>((cfg->ny + TY - 1) / TY));
  kern<<<grid, kThreads, smem, st>>>(in, out, cfg->nx, cfg->ny, periodic, vec_ok, cfg->left,
                                     cfg->right, cfg->top, cfg->bottom, d_w, xform, epi);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

template <typename T, int TY>
int dispatch_spec(int variant, const T* in, T* out, int64_t nx, int64_t ny, int periodic,
                  int vec_ok, const Taps<T>& taps, cudaStream_t st) {
  switch (variant) {
#define CS_SPEC_CASE(I) \
  case I: return launch_spec<T, TY, I>(in, out, nx, ny, periodic, vec_ok, taps, st);
    CS_SPEC_CASE(0) CS_SPEC_CASE(1) CS_SPEC_CASE(2) CS_SPEC_CASE(3) CS_SPEC_CASE(4)
    CS_SPEC_CASE(5) CS_SPEC_CASE(6) CS_SPEC_CASE(7) CS_SPEC_CASE(8) CS_SPEC_CASE(9)
    CS_SPEC_CASE(10) CS_SPEC_CASE(11) CS_SPEC_CASE(12) CS_SPEC_CASE(13)
#undef CS_SPEC_CASE
    default: return set_error(CS_EINVAL, "internal: unknown stencil variant %d", variant);
  }
}
static_assert(kNumSpecs == 14, "update dispatch_spec");

template <typename T>
int launch_stencil2d_t(const Stencil2DConfig* cfg, const void* vin, void* vout, cudaStream_t st) {
  const T* in = static_cast<const T*>(vin);
  T* out = static_cast<T*>(vout);
  const int periodic = cfg->bc == CS_BC_PERIODIC;
  const int vec_ok = (cfg->nx % Vec<T>::n == 0) && (reinterpret_cast<uintptr_t>(in) % 16 == 0);
  if (cfg->variant >= 0) {
    Taps<T> taps;
    const SpecDesc& sd = kSpecs[cfg->variant];
    const int nt = (sd.L + sd.R + 1) * (sd.T + sd.B + 1);
    for (int i = 0; i < 32; ++i) taps.w[i] = i < nt ? static_cast<T>(cfg->weights[i]) : T(0);
    if (cfg->tile_rows == 32)
      return dispatch_spec<T, 32>(cfg->variant, in, out, cfg->nx, cfg->ny, periodic, vec_ok, taps, st);
    return dispatch_spec<T, 64>(cfg->variant, in, out, cfg->nx, cfg->ny, periodic, vec_ok, taps, st);
  }
  const T* d_w;
  if constexpr (sizeof(T) == 8) d_w = reinterpret_cast<const T*>(cfg->d_weights);
  else d_w = reinterpret_cast<const T*>(cfg->d_weights_f);
  const int xform = cfg->fn == CS_FN_CH_NONLIN_LAP, epi = cfg->fn == CS_FN_CUBIC_MINUS_LAP;
  if (cfg->tile_rows == 32)
    return launch_generic<T, 32>(in, out, cfg, d_w, periodic, vec_ok, xform, epi, st);
  return launch_generic<T, 64>(in, out, cfg, d_w, periodic, vec_ok, xform, epi, st);
}

}  // namespace s2d
}  // namespace cs
