// 2D stencil sweep kernels (Sec. 2-4 of arXiv:1902.09931), templated on the storage type.
//
// out[j][i] = sum_{q,p} w[q][p] * in[j - top + q][i - left + p]      (Sec. 3, Sec. 5.2 ordering)
//
// Each CTA (256 threads) owns a TX x TY output tile (TX = 128 floats or 64 doubles: one warp
// spans it).  Its input tile plus halo is staged in shared memory, by cp.async (interior tiles:
// one unrolled 16-byte copy per chunk; edge tiles: the periodic wrap, any number of wraps,
// resolved in the loader, zero fill for non-periodic out-of-grid cells, never read by a written
// output) or by a TMA-pipelined persistent sweep.  Each thread then owns 4 (FP32) or 2 (FP64)
// adjacent columns and walks down its rows in "push" form, every staged row adding its taps to
// the output rows it feeds; outputs leave as 16-byte stores.  FP64 storage is evaluated on the
// FP32 / integer pipes: exact digit sums (integer weight ratios) or double-float arithmetic.
//
// Specialised kernels fix the extents and the non-zero tap mask at compile time (taps with a
// zero weight are skipped, weights live in the kernel-parameter constant bank); the generic
// kernel takes any extents up to CS_MAX_EXTENT at run time.
#pragma once

#include <cuda.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "cs_digits.cuh"
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
__device__ __forceinline__ void cp_async16_s(unsigned smem_addr, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr), "l"(gmem) : "memory");
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
// Interior tile with compile-time shape: warp w copies rows w, w + 8, ...; lane l the 16-byte
// chunks l and l + 32 of each row (a row has 32 to 64 chunks); no loops left after unrolling,
// no bounds or wrap checks, addresses advanced by constant steps.
template <typename T, int ROWS, int COLS>
__device__ __forceinline__ void load_tile_interior(T* s, const T* __restrict__ in, int64_t nx,
                                                   int64_t gy0, int64_t gx0) {
  constexpr int V = Vec<T>::n, NCH = COLS / V, WARPS = kThreads / 32;
  static_assert(NCH >= 32 && NCH <= 64, "one or two chunks per lane and row");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const char* src = reinterpret_cast<const char*>(in + (gy0 + warp) * nx + gx0) + 16 * lane;
  unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(s + warp * COLS)) + 16u * lane;
  const int64_t src_step = static_cast<int64_t>(WARPS) * nx * static_cast<int64_t>(sizeof(T));
  constexpr unsigned kDstStep = WARPS * COLS * sizeof(T);
  const bool second = lane + 32 < NCH;
#pragma unroll
  for (int k = 0; k < (ROWS + WARPS - 1) / WARPS; ++k) {
    if (k * WARPS + warp < ROWS) {
      cp_async16_s(dst, src);
      if (second) cp_async16_s(dst + 512u, src + 512);
    }
    src += src_step;
    dst += kDstStep;
  }
  cp_async_wait_all();
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void load_tile(T* s, const T* __restrict__ in, int64_t nx, int64_t ny,
                                          bool periodic, bool vec_ok, int64_t x0, int64_t y0,
                                          int top, int LA, int cols, int rows) {
  constexpr int V = Vec<T>::n;
  const int nch = cols / V;
  const int total = rows * nch;
  const int64_t gy0 = y0 - top, gx0 = x0 - LA;
  if (vec_ok && gy0 >= 0 && gy0 + rows <= ny && gx0 >= 0 && gx0 + cols <= nx) {
    // interior tile (the common case): warp w copies rows w, w + 8, ...; lane l the 16-byte
    // chunks l, l + 32, ...; no bounds or wrap checks, addresses advanced by constant steps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const char* src = reinterpret_cast<const char*>(in + (gy0 + warp) * nx + gx0) + 16 * lane;
    unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(s + warp * cols)) + 16u * lane;
    const int64_t src_step = static_cast<int64_t>(kThreads / 32) * nx * static_cast<int64_t>(sizeof(T));
    const unsigned dst_step = static_cast<unsigned>((kThreads / 32) * cols * sizeof(T));
#pragma unroll 4
    for (int r = warp; r < rows; r += kThreads / 32) {
      for (int ch = lane; ch < nch; ch += 32) cp_async16_s(dst + 16u * (ch - lane), src + 16 * (ch - lane));
      src += src_step;
      dst += dst_step;
    }
    cp_async_wait_all();
    __syncthreads();
    return;
  }
  const bool one_wrap = nx >= cols && ny >= rows;  // tile halo reaches at most one period out
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
      gy = one_wrap ? (gy < 0 ? gy + ny : gy - ny) : wrap_idx(gy, ny);
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
          gx = one_wrap ? (gx < 0 ? gx + nx : gx - nx) : wrap_idx(gx, nx);
        }
        cp_async_elem(dst + e, row + gx);
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
}

// load_tile for a compile-time tile shape: interior tiles take the unrolled copy.
template <typename T, int ROWS, int COLS>
__device__ __forceinline__ void load_tile_ct(T* s, const T* __restrict__ in, int64_t nx, int64_t ny,
                                             bool periodic, bool vec_ok, int64_t x0, int64_t y0,
                                             int top, int LA) {
  const int64_t gy0 = y0 - top, gx0 = x0 - LA;
  if (vec_ok && gy0 >= 0 && gy0 + ROWS <= ny && gx0 >= 0 && gx0 + COLS <= nx) {
    load_tile_interior<T, ROWS, COLS>(s, in, nx, gy0, gx0);
    return;
  }
  load_tile<T>(s, in, nx, ny, periodic, vec_ok, x0, y0, top, LA, COLS, ROWS);
}

template <typename T>
__device__ __forceinline__ void xform_tile(T* s, int n) {
  for (int i = threadIdx.x; i < n; i += kThreads) s[i] = cubic_minus(s[i]);
  __syncthreads();
}

// FP32 compute phase of the specialised kernels: each thread owns four adjacent columns of the
// tile (one warp spans its 128 columns) and walks down its rows in "push" form: every staged row
// adds its taps to the (up to H) output rows it feeds, in the tap order (row, column) of a
// one-output evaluation, so each output is the same chain of FMAs.  Rows are read as 16-byte
// column groups and the four results leave as one 16-byte store where all four are written.
template <int TY, int SPEC>
__device__ __forceinline__ void spec_compute_f32(const float* s, float* __restrict__ out, int64_t nx,
                                                 int64_t ny, int periodic, int64_t x0, int64_t y0,
                                                 const Taps<float>& taps) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int L = sd.L, R = sd.R, TT = sd.T, BB = sd.B;
  constexpr int TX = tile_x<float>();
  static_assert(TX == 128, "one warp spans the tile's 128 columns");
  constexpr int LA = (L + 3) / 4 * 4, RA = (R + 3) / 4 * 4;
  constexpr int COLS = LA + TX + RA, C4 = COLS / 4;
  constexpr int W = L + R + 1, H = TT + BB + 1;
  constexpr int WY = kThreads / 32, RW = TY / WY;
  constexpr int NC = LA / 4 + 1 + (3 + R) / 4;  // 16-byte groups read per row
  constexpr int OFF = LA - L;                   // window index of tap p for column j: OFF + j + p
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = 4 * lane;
  const int r0 = warp * RW;
  const int64_t gx = x0 + c;
  bool ok[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) ok[j] = gx + j < nx && (periodic || (gx + j >= L && gx + j < nx - R));
  const bool any = ok[0] || ok[1] || ok[2] || ok[3];
  const bool all4 = ok[0] && ok[1] && ok[2] && ok[3] && (reinterpret_cast<uintptr_t>(out) & 15u) == 0 &&
                    (nx & 3) == 0;
  const int64_t gy0 = y0 + r0;
  const int64_t ylo = periodic ? 0 : TT, yhi = periodic ? ny : ny - BB;
  auto rows_below = [](int64_t d) { return static_cast<int>(d < 0 ? 0 : (d > RW ? RW : d)); };
  const int klo = rows_below(ylo - gy0);
  const int khi = any ? rows_below(yhi - gy0) : 0;
  float* op = out + gy0 * nx + gx;
  const float4* a = reinterpret_cast<const float4*>(s) + lane;  // window starts at smem column c
  float acc[H][4];
#pragma unroll
  for (int q = 0; q < H; ++q)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[q][j] = 0.0f;
#pragma unroll
  for (int i = 0; i < RW + H - 1; ++i) {
    float x[4 * NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      bool used = false;
#pragma unroll
      for (int q = 0; q < H; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int p = 0; p < W; ++p)
            used |= (OFF + j + p) / 4 == k && ((sd.mask >> (q * W + p)) & 1u) && (i - q >= 0) && (i - q < RW);
      if (used) {
        const float4 v = a[(r0 + i) * C4 + k];
        x[4 * k] = v.x;
        x[4 * k + 1] = v.y;
        x[4 * k + 2] = v.z;
        x[4 * k + 3] = v.w;
      }
    }
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const int o = i - q;
      if (o < 0 || o >= RW) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int p = 0; p < W; ++p)
          if ((sd.mask >> (q * W + p)) & 1u) acc[o % H][j] = fmaf(taps.w[q * W + p], x[OFF + j + p], acc[o % H][j]);
    }
    const int done = i - (H - 1);
    if (done >= 0) {
      float* r = acc[done % H];
      if constexpr (sd.epi) {
        const float4 u = reinterpret_cast<const float4*>(s)[(r0 + done + TT) * C4 + lane + LA / 4];
        r[0] = cubic_minus(u.x) + r[0];
        r[1] = cubic_minus(u.y) + r[1];
        r[2] = cubic_minus(u.z) + r[2];
        r[3] = cubic_minus(u.w) + r[3];
      }
      if (done >= klo && done < khi) {
        if (all4) {
          *reinterpret_cast<float4*>(op) = make_float4(r[0], r[1], r[2], r[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (ok[j]) op[j] = r[j];
        }
      }
      r[0] = r[1] = r[2] = r[3] = 0.0f;
      op += nx;
    }
  }
}

// Compute phase of the specialised kernels in the storage type: each thread owns one column
// of the tile and walks down its rows with a register window; `s` is the staged tile.
template <typename T, int TY, int SPEC>
__device__ __forceinline__ void spec_compute(const T* s, T* __restrict__ out, int64_t nx,
                                             int64_t ny, int periodic, int64_t x0, int64_t y0,
                                             const Taps<T>& taps) {
  if constexpr (sizeof(T) == 4) {
    spec_compute_f32<TY, SPEC>(s, out, nx, ny, periodic, x0, y0, taps);
    return;
  }
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int L = sd.L, R = sd.R, TT = sd.T, BB = sd.B;
  constexpr int V = Vec<T>::n;
  constexpr int TX = tile_x<T>();
  constexpr int LA = (L + V - 1) / V * V, RA = (R + V - 1) / V * V;
  constexpr int COLS = LA + TX + RA;
  constexpr int W = L + R + 1, H = TT + BB + 1;
  constexpr int WX = TX / 32, WY = 8 / WX, RW = TY / WY;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = (warp % WX) * 32 + lane;
  const int r0 = (warp / WX) * RW;
  const int64_t gx = x0 + c;
  const bool col_ok = gx < nx && (periodic || (gx >= L && gx < nx - R));
  // this thread writes rows gy0 + k for klo <= k < khi of its column
  const int64_t gy0 = y0 + r0;
  const int64_t ylo = periodic ? 0 : TT, yhi = periodic ? ny : ny - BB;
  auto rows_below = [](int64_t d) { return static_cast<int>(d < 0 ? 0 : (d > RW ? RW : d)); };
  const int klo = rows_below(ylo - gy0);
  const int khi = col_ok ? rows_below(yhi - gy0) : 0;
  T* op = out + gy0 * nx + gx;
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
    if (k >= klo && k < khi) *op = acc;
    op += nx;
  }
}

template <typename T, int TY, int SPEC>
__global__ void __launch_bounds__(kThreads)
    k_stencil2d_spec(const T* __restrict__ in, T* __restrict__ out, int64_t nx, int64_t ny,
                     int periodic, int vec_ok, Taps<T> taps, int ty0) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int V = Vec<T>::n;
  constexpr int TX = tile_x<T>();
  constexpr int LA = (sd.L + V - 1) / V * V, RA = (sd.R + V - 1) / V * V;
  constexpr int COLS = LA + TX + RA, ROWS = TY + sd.T + sd.B;
  static_assert((sd.L + sd.R + 1) * (sd.T + sd.B + 1) <= 32, "tap table too small");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * TX;
  const int64_t y0 = (static_cast<int64_t>(blockIdx.y) + ty0) * TY;
  load_tile_ct<T, ROWS, COLS>(s, in, nx, ny, periodic != 0, vec_ok != 0, x0, y0, sd.T, LA);
  if constexpr (sd.xform) xform_tile<T>(s, ROWS * COLS);
  spec_compute<T, TY, SPEC>(s, out, nx, ny, periodic, x0, y0, taps);
}

template <typename T>
inline size_t tile_smem_bytes(int L, int R, int TT, int BB, int TY, bool generic) {
  constexpr int V = Vec<T>::n;
  const int LA = (L + V - 1) / V * V, RA = (R + V - 1) / V * V;
  size_t b = sizeof(T) * static_cast<size_t>(TY + TT + BB) * (LA + tile_x<T>() + RA);
  if (generic) b += sizeof(T) * static_cast<size_t>((L + R + 1) * (TT + BB + 1));
  return b;
}

// The double-float steps run packed (FP32x2) over two adjacent output columns: lane x is the left
// column, y the right; each lane rounds exactly as a scalar evaluation would.  a - b is formed as
// fma(b, -1, a) (one rounding, as a subtraction).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, f2(-1.0f)); }

// (sh, sl) += (wh + wl) * (xh + xl): the product's rounding error comes from an FMA and the sum
// is an error-free TwoSum; the wl * xl term (~2^-48 relative) is dropped.
__device__ __forceinline__ void dd_mac2(float2& sh, float2& sl, float wh, float wl, float2 xh, float2 xl) {
  const float2 q = __fmul2_rn(f2(-wh), xh);  // q = -p, p = wh * xh rounded
  float2 e = __ffma2_rn(f2(wh), xh, q);      // exact: wh * xh - p
  e = __ffma2_rn(f2(wh), xl, e);
  e = __ffma2_rn(f2(wl), xh, e);
  const float2 s = sub2(sh, q);              // TwoSum(sh, p)
  const float2 bb = sub2(s, sh);
  const float2 err = sub2(sub2(sh, sub2(s, bb)), __fadd2_rn(q, bb));  // (sh - (s - bb)) + (p - bb)
  sl = __fadd2_rn(sl, __fadd2_rn(err, e));
  sh = s;
}

// (sh, sl) += p + e with an error-free TwoSum of sh and p.
__device__ __forceinline__ void dd_add_exact2(float2& sh, float2& sl, float2 p, float2 e) {
  const float2 s = __fadd2_rn(sh, p);
  const float2 bb = sub2(s, sh);
  const float2 err = __fadd2_rn(sub2(sh, sub2(s, bb)), sub2(p, bb));
  sl = __fadd2_rn(sl, __fadd2_rn(err, e));
  sh = s;
}

// (sh, sl) += u^3 - u for u = uh + ul, with error-free products and sums (terms below ~2^-46
// of |u| dropped), so the cubic of the user function stays on the FP32 pipes.
__device__ __forceinline__ void dd_add_cubic_minus2(float2& sh, float2& sl, float2 uh, float2 ul) {
  const float2 p2 = __fmul2_rn(uh, uh);  // u^2 = p2 + e2
  float2 e2 = __ffma2_rn(uh, uh, neg2(p2));
  e2 = __ffma2_rn(__fmul2_rn(f2(2.0f), uh), ul, e2);
  const float2 p3 = __fmul2_rn(p2, uh);  // u^3 = p3 + e3
  float2 e3 = __ffma2_rn(p2, uh, neg2(p3));
  e3 = __ffma2_rn(p2, ul, e3);
  e3 = __ffma2_rn(e2, uh, e3);
  dd_add_exact2(sh, sl, p3, e3);
  dd_add_exact2(sh, sl, neg2(uh), neg2(ul));
}

// ---- exact digit evaluation of FP64-storage stencils with integer weight ratios ------------
// When every weight is w_k = c * n_k with small integers (sum |n_k| <= 64; the paper's stencils
// are of this kind), a tile is evaluated with integer-exact sums: every staged value is cut into
// two 24-bit integer digits (d0 signed, 0 <= d1 < 2^24) on a grid fixed by the tile's largest exponent,
// x = (d0 2^24 + d1) 2^(G-48) + r with |r| < 2^(G-48), so each digit sum S_i = sum_k n_k d_{k,i}
// is exact in int32 (per tap two integer multiply-adds).  The sums form T = S0 2^24 + S1, which is
// rounded to a multiple of 2^4 and scaled by c * 2^(G-48) with one FP64 FMA (ixi_combine).  The
// error is at most (2^-47 + 2^-44 / sum|n| + 2^-50) of sum|w| * max|in| (native FP64 accumulation: about
// taps * 2^-53 of sum|w| |in|).  Tiles holding inf / nan, or whose largest value is outside
// [2^-900, 2^900], are evaluated in native FP64.

struct IxTaps {
  int8_t n[32];  // integer weight ratios n_k (sum |n_k| <= 64)
  double c;      // common scale, w_k ~= c * n_k, rounded to 51 bits (ixi_round51)
  double c15;    // -1.5 c (exact)
  float inv_hi, inv_lo;  // 1 / c as a float pair (the user function's cubic term)
};

// The user function c^3 - c + sum w_k u_k (Sec. 5.2, variant 13) on the digit path: the cubic
// term P = u^3 - u of the centre value, in double-float arithmetic from the value's digits, joins
// the digit sum as the integer Q = round(P / U) in units U = c 2^(G-44) of the combination, so the
// output is still rounded once by the one FP64 FMA.  Valid when |P / U| < 2^43, which holds when
// |c| >= 4 (the host's condition) and 2G <= e_c - 2 (e_c = floor(log2 |c|), |u| < 2^G), with the
// tile's values in the double-float exponent range; other tiles take native FP64.  Q's error is
// below one unit U (the truncated digits, the double-float cubic and product, ~2^-46 relative).
__device__ __forceinline__ bool ixf_tile_ok(int tile_e, double c) {
  if (tile_e == 0) return true;
  const int G = tile_e - 1022;
  const int ec = static_cast<int>((static_cast<uint32_t>(__double2hiint(c)) >> 20) & 0x7ffu) - 1023;
  return tile_e >= 1023 - 69 && tile_e < 1023 + 60 && 2 * G <= ec - 2;
}

// Per-tile constants of the cubic term: 2^(G-24), 2^(G-48) (digit weights) and (1/c) 2^(44-G) as
// a float pair, by adding to the exponent fields (all stay normal in the tile's valid range).
struct IxfConsts { float p1, p2, ih, il; };
__device__ __forceinline__ IxfConsts ixf_consts(int tile_e, float inv_hi, float inv_lo) {
  const int G = tile_e - 1022;
  IxfConsts k;
  k.p1 = __uint_as_float(static_cast<uint32_t>(G - 24 + 127) << 23);
  k.p2 = __uint_as_float(static_cast<uint32_t>(G - 48 + 127) << 23);
  const uint32_t shift = static_cast<uint32_t>(44 - G) << 23;
  k.ih = __uint_as_float(__float_as_uint(inv_hi) + shift);
  k.il = inv_lo == 0.0f ? 0.0f : __uint_as_float(__float_as_uint(inv_lo) + shift);
  return k;
}

// Q for the centre digits (d0, d1) of two adjacent outputs (packed FP32x2), returned as
// Q = qa 2^20 + qb (the split ixi_combine takes).  u = uh + ul with uh = d0 2^(G-24) and
// ul = d1 2^(G-48) (both exact floats); P = u^3 - u in double-float with error-free products and
// sums, carried negated where that saves a negation (a packed FMA has no free operand sign):
// m2 = -uh^2 rounded, u^2 = -m2 + e2; m3 = m2 uh = -(p2 uh) rounded, u^3 = -m3 + e3; then
// -P = (m3 + uh) + (ul - e3), summed with TwoSum into s + lo.  R = -P (1/c) 2^(44-G) =
// (s + lo)(ih + il) is formed as -nph + pl and renormalised with Fast2Sum to qh + ql
// (|ql| <= half an ulp of qh).  round(qh + ql) comes from two FP32 rounding shifts:
// 1.5 * 2^44 takes qh to a multiple of 2^21 (|qh| < 2^43), whose count k sits in the low mantissa
// bits, and 1.5 * 2^23 rounds the rest (|rest| < 2^22) to k2; Q = -(k 2^21 + k2), so
// qa = -2k and qb = -k2 (ties to even is symmetric).  The only conversions are the four exact
// int -> float conversions of the digits.
__device__ __forceinline__ void ixf_q2(int2 a, int2 b, const IxfConsts& k, int2& qa, int2& qb) {
  const float2 D0 = make_float2(__int2float_rn(a.x), __int2float_rn(b.x));
  const float2 D1 = make_float2(__int2float_rn(a.y), __int2float_rn(b.y));
  const float2 uh = __fmul2_rn(D0, f2(k.p1));
  const float2 nuh = __fmul2_rn(D0, f2(-k.p1));
  const float2 ul = __fmul2_rn(D1, f2(k.p2));
  const float2 nul = __fmul2_rn(D1, f2(-k.p2));
  const float2 m2 = __fmul2_rn(nuh, uh);
  float2 e2 = __ffma2_rn(uh, uh, m2);
  e2 = __ffma2_rn(__fmul2_rn(D0, f2(2.0f * k.p1)), ul, e2);
  const float2 m3 = __fmul2_rn(m2, uh);
  float2 e3 = __ffma2_rn(m2, nuh, m3);
  e3 = __ffma2_rn(m2, nul, e3);
  e3 = __ffma2_rn(e2, uh, e3);
  const float2 s = __fadd2_rn(m3, uh);  // TwoSum(m3, uh)
  const float2 bb = sub2(s, m3);
  const float2 err = __fadd2_rn(sub2(m3, sub2(s, bb)), sub2(uh, bb));
  const float2 lo = __fadd2_rn(sub2(err, e3), ul);
  const float2 nph = __fmul2_rn(s, f2(-k.ih));
  float2 pl = __ffma2_rn(s, f2(k.ih), nph);
  pl = __ffma2_rn(lo, f2(k.ih), pl);
  pl = __ffma2_rn(s, f2(k.il), pl);
  const float2 qh = sub2(pl, nph);  // Fast2Sum(-nph, pl)
  const float2 ql = sub2(pl, __fadd2_rn(qh, nph));
  constexpr float M1 = 26388279066624.0f, M2 = 12582912.0f;  // 1.5 * 2^44, 1.5 * 2^23
  const float2 t = __fadd2_rn(qh, f2(M1));
  const float2 rest = __fadd2_rn(sub2(qh, sub2(t, f2(M1))), ql);
  const float2 t2 = __fadd2_rn(rest, f2(M2));
  qa = make_int2(2 * static_cast<int>(__float_as_uint(M1) - __float_as_uint(t.x)),
                 2 * static_cast<int>(__float_as_uint(M1) - __float_as_uint(t.y)));
  qb = make_int2(static_cast<int>(__float_as_uint(M2) - __float_as_uint(t2.x)),
                 static_cast<int>(__float_as_uint(M2) - __float_as_uint(t2.y)));
}

using ixd::ixi_combine;
using ixd::ixi_consts;

// Compile-time weight ratios of the digit sums (CW = 2): the 5-point pattern of the user function
// c^3 - c - Lap c, whose ratios the plan always sets to (0, -1, 0, -1, 4, -1, 0, -1, 0); the
// compiler then forms the sum from adds and one shift instead of an integer multiply-add per tap.
// Every other stencil takes the plan's ratios (CW = 0).
template <int CW>
__device__ __forceinline__ int ix_weight(const IxTaps& taps, int k) {
  if constexpr (CW == 2) {  // 3 x 3 footprint, k = row * 3 + column
    return k == 4 ? 4 : (k == 1 || k == 3 || k == 5 || k == 7) ? -1 : 0;
  } else {
    return static_cast<int>(taps.n[k]);
  }
}

// Digit sums of two adjacent tile columns per thread, "push" form: every staged row adds its
// contributions to the (up to H) output rows it feeds, held in H rolling accumulators per column
// and digit; an output row is complete once its last input row has been added.  A row's digits
// are read as 16-byte (d0, d1, d0', d1') pairs of columns, W + 1 columns (+1 when L is odd)
// serving both outputs, and the two results leave as one 16-byte store where both columns are
// written.
// FULL: every output of the tile is written and 16-byte stores apply (the launch checked that the
// grid is periodic, nx a multiple of 64, ny of TY, and out 16-byte aligned); the per-row range and
// alignment tests are left out.
template <int TY, int SPEC, bool FULL = false, int CW = 0>
__device__ __forceinline__ void ix_compute(const int2* sd2, double* __restrict__ out, int64_t nx,
                                           int64_t ny, int periodic, int64_t x0, int64_t y0,
                                           const IxTaps& taps, const uint32_t (&w)[4], int tile_e) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int L = sd.L, R = sd.R, TT = sd.T, BB = sd.B;
  constexpr int V = Vec<double>::n;
  constexpr int TX = tile_x<double>();
  static_assert(TX == 64, "one warp spans the tile's 64 columns");
  constexpr int LA = (L + V - 1) / V * V, RA = (R + V - 1) / V * V;
  constexpr int COLS = LA + TX + RA;
  constexpr int W = L + R + 1, H = TT + BB + 1;
  constexpr int WY = kThreads / 32, RW = TY / WY;
  constexpr int S0 = LA - L, X = S0 & 1, NP = (W + 1 + X + 1) / 2;  // pairs read per row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = 2 * lane;
  const int r0 = warp * RW;
  const int64_t gx = x0 + c;
  const bool ok0 = gx < nx && (periodic || (gx >= L && gx < nx - R));
  const bool ok1 = gx + 1 < nx && (periodic || (gx + 1 >= L && gx + 1 < nx - R));
  // one 16-byte store per row when both columns are written and every row start is 16-byte aligned
  const bool both = ok0 && ok1 && (reinterpret_cast<uintptr_t>(out) & 15u) == 0 && (nx & 1) == 0;
  // this thread writes rows gy0 + k for klo <= k < khi
  const int64_t gy0 = y0 + r0;
  const int64_t ylo = periodic ? 0 : TT, yhi = periodic ? ny : ny - BB;
  auto rows_below = [](int64_t d) { return static_cast<int>(d < 0 ? 0 : (d > RW ? RW : d)); };
  const int klo = rows_below(ylo - gy0);
  const int khi = (ok0 || ok1) ? rows_below(yhi - gy0) : 0;
  double* op = out + gy0 * nx + gx;
  const int4* a = reinterpret_cast<const int4*>(sd2 + (S0 - X) + c);  // (S0 - X + c) is even
  int acc0[H][2], acc1[H][2];
#pragma unroll
  for (int q = 0; q < H; ++q)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc0[q][j] = acc1[q][j] = 0;
  // user function: the centre digits of the pending output rows, and the per-tile constants
  int2 ctr[H][2];
  IxfConsts kf{};
  if constexpr (sd.epi) {
    if (tile_e != 0) kf = ixf_consts(tile_e, taps.inv_hi, taps.inv_lo);
  }
#pragma unroll
  for (int i = 0; i < RW + H - 1; ++i) {  // input row r0 + i feeds output rows i - q
    int2 v[2 * NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      bool used = false;
#pragma unroll
      for (int q = 0; q < H; ++q)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int p = 0; p < W; ++p) {
            const int e = X + j + p;
            used |= (e >> 1) == k && ((sd.mask >> (q * W + p)) & 1u) && (i - q >= 0) && (i - q < RW);
          }
      if (used) {
        const int4 d = a[(r0 + i) * (COLS / 2) + k];
        v[2 * k] = make_int2(d.x, d.y);
        v[2 * k + 1] = make_int2(d.z, d.w);
      }
    }
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const int o = i - q;
      if (o < 0 || o >= RW) continue;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
#pragma unroll
        for (int p = 0; p < W; ++p)
          if ((sd.mask >> (q * W + p)) & 1u) {
            const int n = ix_weight<CW>(taps, q * W + p);
            acc0[o % H][j] += n * v[X + j + p].x;
            acc1[o % H][j] += n * v[X + j + p].y;
          }
      }
    }
    if constexpr (sd.epi) {  // this row is the centre row of output row i - TT
      if (i - TT >= 0 && i - TT < RW) {
        ctr[(i - TT) % H][0] = v[X + L];
        ctr[(i - TT) % H][1] = v[X + 1 + L];
      }
    }
    const int done = i - (H - 1);  // output row complete after its last input row
    if (done >= 0) {
      int2 qa = make_int2(0, 0), qb = make_int2(0, 0);
      if constexpr (sd.epi) {
        ixf_q2(ctr[done % H][0], ctr[done % H][1], kf, qa, qb);  // kf is all zero for a zero tile: Q = 0
      }
      const double val0 = ixi_combine(acc0[done % H][0], acc1[done % H][0], w, qa.x, qb.x);
      const double val1 = ixi_combine(acc0[done % H][1], acc1[done % H][1], w, qa.y, qb.y);
      acc0[done % H][0] = acc0[done % H][1] = acc1[done % H][0] = acc1[done % H][1] = 0;
      if constexpr (FULL) {
        *reinterpret_cast<double2*>(op) = make_double2(val0, val1);
      } else if (done >= klo && done < khi) {
        if (both) {
          *reinterpret_cast<double2*>(op) = make_double2(val0, val1);
        } else {
          if (ok0) op[0] = val0;
          if (ok1) op[1] = val1;
        }
      }
      op += nx;
    }
  }
}

// Resident CTAs of the digit kernel: at least 6 (40 registers per thread, 48 warps per SM; the
// tile's shared memory allows 6) for footprints of at most 13 taps over at most 5 rows, whose
// rolling digit sums fit that budget; at least 3 (85 registers) for the larger footprints.  More
// resident CTAs let one CTA's load and reduction phases overlap the others' digit sums.
constexpr int ix_min_blocks(int spec) {
  int taps = 0;
  for (unsigned m = kSpecs[spec].mask; m != 0u; m &= m - 1u) ++taps;
  return kSpecs[spec].T + kSpecs[spec].B + 1 <= 5 && taps <= 13 ? 6 : 3;
}

template <int TY, int SPEC, bool FULL, int CW = 0>
__global__ void __launch_bounds__(kThreads, ix_min_blocks(SPEC))
    k_stencil2d_ix(const double* __restrict__ in, double* __restrict__ out, int64_t nx, int64_t ny,
                   int periodic, int vec_ok, Taps<double> taps, IxTaps itaps, int tx0, int ty0, int ring_nbx,
                   int ring_nby) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int V = Vec<double>::n;
  constexpr int TX = tile_x<double>();
  constexpr int LA = (sd.L + V - 1) / V * V, RA = (sd.R + V - 1) / V * V;
  constexpr int COLS = LA + TX + RA, ROWS = TY + sd.T + sd.B;
  static_assert(!sd.xform, "digit kernel covers weighted stencils and the cubic user function");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s = reinterpret_cast<double*>(smem_raw);
  __shared__ __align__(16) unsigned s_red[kThreads / 32];
  static_assert(COLS % 2 == 0, "digit passes take values in pairs");
  // the tile: (blockIdx.x + tx0, blockIdx.y + ty0), or with ring_nbx > 0 the CTA's tile of the
  // border ring of an nbx x nby tile grid (the top row, the bottom row, then the first and last
  // columns of the rows between)
  int64_t bx = static_cast<int64_t>(blockIdx.x) + tx0, by = static_cast<int64_t>(blockIdx.y) + ty0;
  if (ring_nbx > 0) {
    const int b = static_cast<int>(blockIdx.x), mid = ring_nby - 2;
    if (b < ring_nbx) {
      bx = b;
      by = 0;
    } else if (b < 2 * ring_nbx) {
      bx = b - ring_nbx;
      by = ring_nby - 1;
    } else {
      const int c = b - 2 * ring_nbx, side = c / mid;
      bx = side ? ring_nbx - 1 : 0;
      by = 1 + (c - side * mid);
    }
  }
  const int64_t x0 = bx * TX;
  const int64_t y0 = by * TY;
  load_tile_ct<double, ROWS, COLS>(s, in, nx, ny, periodic != 0, vec_ok != 0, x0, y0, sd.T, LA);
  // pass 1: the tile's largest exponent; inf / nan (and tiles outside the exponent window) take
  // native FP64
  const uint32_t mhi = ixd::ix_tile_max_hi<kThreads, ROWS * COLS>(s, s_red);
  const int tile_e = static_cast<int>(mhi >> 20);
  uint32_t w[4];
  if (!ixi_consts(itaps.c, itaps.c15, tile_e, w) || (sd.epi && !ixf_tile_ok(tile_e, itaps.c))) {
    spec_compute<double, TY, SPEC>(s, out, nx, ny, periodic, x0, y0, taps);
    return;
  }
  // pass 2: integer digits over the values' own slots
  ixd::ixi_split_tile<kThreads, ROWS * COLS>(s, tile_e);
  __syncthreads();
  ix_compute<TY, SPEC, FULL, CW>(reinterpret_cast<const int2*>(s), out, nx, ny, periodic, x0, y0, itaps, w, tile_e);
}

// Output rows [row0, row1) of the next launches on this host thread (row0 a multiple of 64, so
// of every tile height; row1 < 0: to the last row).  Set by stencil2d_launch_rows for the banded
// host-buffer path; every other launch covers the whole grid.
struct RowWindow { int64_t row0 = 0, row1 = -1; };
inline RowWindow& row_window() {
  static thread_local RowWindow w;
  return w;
}
// First tile row and number of tile rows of height ty that the window covers in a grid of ny rows.
inline void window_tiles(int ty, int64_t ny, int* ty0, int* nty) {
  const RowWindow& w = row_window();
  const int64_t r1 = w.row1 < 0 || w.row1 > ny ? ny : w.row1;
  const int64_t t0 = w.row0 / ty, t1 = (r1 + ty - 1) / ty;
  *ty0 = static_cast<int>(t0);
  *nty = static_cast<int>(t1 > t0 ? t1 - t0 : 0);
}

template <int TY, int SPEC>
int launch_ix(const double* in, double* out, int64_t nx, int64_t ny, int periodic, int vec_ok,
              const Taps<double>& taps, const IxTaps& itaps, const Stencil2DConfig* cfg, cudaStream_t st) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int TX = tile_x<double>();
  const size_t smem = tile_smem_bytes<double>(sd.L, sd.R, sd.T, sd.B, TY, false);
  // the cubic user function's fixed ratios are compiled in (ix_weight)
  constexpr int CWS = SPEC == 13 ? 2 : 0;
  auto kfull = k_stencil2d_ix<TY, SPEC, true, CWS>;
  auto kedge = k_stencil2d_ix<TY, SPEC, false, CWS>;
  static bool attr_set = false;
  if (!attr_set) {
    CS_CUDA_TRY(cudaFuncSetAttribute(kfull, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    CS_CUDA_TRY(cudaFuncSetAttribute(kedge, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    attr_set = true;
  }
  int ty0, nty;
  window_tiles(TY, ny, &ty0, &nty);
  if (nty == 0) return CS_OK;
  const int64_t nbx = (nx + TX - 1) / TX, nby = (ny + TY - 1) / TY;
  // the FULL form (every output of a tile written, 16-byte stores) applies to every tile of a
  // periodic grid of whole tiles, and to the inner tiles of a non-periodic one
  const bool whole = nx % TX == 0 && ny % TY == 0 && (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  if (periodic || !whole || !cfg || !cfg->aux || ty0 != 0 || nty != nby || nbx < 3 || nby < 3) {
    auto kern = periodic && whole ? kfull : kedge;
    dim3 grid(static_cast<unsigned>(nbx), static_cast<unsigned>(nty));
    kern<<<grid, kThreads, smem, st>>>(in, out, nx, ny, periodic, vec_ok, taps, itaps, 0, ty0, 0, 0);
    CS_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return CS_OK;
  }
  // non-periodic: the border ring of tiles (the general form) on the plan's second stream, beside
  // the inner tiles (FULL) on st; st then waits for both
  CS_CUDA_TRY(cudaEventRecord(cfg->ev_fork, st));
  CS_CUDA_TRY(cudaStreamWaitEvent(cfg->aux, cfg->ev_fork, 0));
  const unsigned nring = static_cast<unsigned>(2 * nbx + 2 * (nby - 2));
  kedge<<<nring, kThreads, smem, cfg->aux>>>(in, out, nx, ny, periodic, vec_ok, taps, itaps, 0, 0,
                                             static_cast<int>(nbx), static_cast<int>(nby));
  CS_CUDA_TRY(cudaGetLastError());
  CS_CUDA_TRY(cudaEventRecord(cfg->ev_join, cfg->aux));
  dim3 grid(static_cast<unsigned>(nbx - 2), static_cast<unsigned>(nby - 2));
  kfull<<<grid, kThreads, smem, st>>>(in, out, nx, ny, periodic, vec_ok, taps, itaps, 1, 1, 0, 0);
  CS_CUDA_TRY(cudaGetLastError());
  CS_CUDA_TRY(cudaStreamWaitEvent(st, cfg->ev_join, 0));
  count_launches(2);
  return CS_OK;
}

template <int TY>
int dispatch_ix(int variant, const double* in, double* out, int64_t nx, int64_t ny, int periodic,
                int vec_ok, const Taps<double>& taps, const IxTaps& itaps, const Stencil2DConfig* cfg,
                cudaStream_t st) {
  switch (variant) {
#define CS_IX_CASE(I) \
  case I: return launch_ix<TY, I>(in, out, nx, ny, periodic, vec_ok, taps, itaps, cfg, st);
    CS_IX_CASE(0) CS_IX_CASE(1) CS_IX_CASE(2) CS_IX_CASE(3) CS_IX_CASE(4)
    CS_IX_CASE(5) CS_IX_CASE(6) CS_IX_CASE(7) CS_IX_CASE(8) CS_IX_CASE(9)
    CS_IX_CASE(10) CS_IX_CASE(11) CS_IX_CASE(13)
#undef CS_IX_CASE
    default: return set_error(CS_EINVAL, "internal: variant %d has no digit kernel", variant);
  }
}

// ---- grouped launch: several independent grids, one persistent kernel ---------------------
// The job table travels as a __grid_constant__ kernel parameter (kept in the constant bank,
// indexable without a local copy; up to kMaxGroup jobs per launch).  The grid is sized to the
// resident CTAs of the GPU; CTA b walks the tiles b, b + gridDim.x, ... of all jobs in order,
// advancing its job index as the tile index passes each job's range, and evaluates each tile as
// the specialised kernel does: storage-type arithmetic (MODE 0), or for FP64 storage the exact
// digit path (MODE 1, every job's weights integer ratios; tiles out of its range take native
// FP64).  Nothing is allocated and nothing synchronises, so a grouped launch can be captured in a
// CUDA graph.
constexpr int kMaxGroup = 64;

template <typename T> struct GroupJob {
  const T* in;
  T* out;
  int64_t nx, ny;
  int tiles_x, tile_begin, periodic, vec_ok;
  Taps<T> taps;
  IxTaps itaps;
};
template <typename T> struct GroupTable {
  int count, total_tiles;
  GroupJob<T> job[kMaxGroup];
};

template <typename T, int TY, int SPEC, int MODE>
__global__ void __launch_bounds__(kThreads) k_stencil2d_group(const __grid_constant__ GroupTable<T> tab) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int V = Vec<T>::n;
  constexpr int TX = tile_x<T>();
  constexpr int LA = (sd.L + V - 1) / V * V, RA = (sd.R + V - 1) / V * V;
  constexpr int COLS = LA + TX + RA, ROWS = TY + sd.T + sd.B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) unsigned s_red[kThreads / 32];
  T* s = reinterpret_cast<T*>(smem_raw);
  int j = 0;
  for (int b = static_cast<int>(blockIdx.x); b < tab.total_tiles; b += static_cast<int>(gridDim.x)) {
    while (j + 1 < tab.count && b >= tab.job[j + 1].tile_begin) ++j;
    const GroupJob<T>& g = tab.job[j];
    const int t = b - g.tile_begin;
    const int64_t x0 = static_cast<int64_t>(t % g.tiles_x) * TX;
    const int64_t y0 = static_cast<int64_t>(t / g.tiles_x) * TY;
    __syncthreads();  // the previous tile's reads of s are done
    load_tile_ct<T, ROWS, COLS>(s, g.in, g.nx, g.ny, g.periodic != 0, g.vec_ok != 0, x0, y0, sd.T, LA);
    if constexpr (MODE == 1 && !sd.xform && sizeof(T) == 8) {
      const uint32_t mhi = ixd::ix_tile_max_hi<kThreads, ROWS * COLS>(s, s_red);
      const int tile_e = static_cast<int>(mhi >> 20);
      uint32_t w[4];
      if (!ixi_consts(g.itaps.c, g.itaps.c15, tile_e, w) || (sd.epi && !ixf_tile_ok(tile_e, g.itaps.c))) {
        spec_compute<double, TY, SPEC>(s, g.out, g.nx, g.ny, g.periodic, x0, y0, g.taps);
      } else {
        ixd::ixi_split_tile<kThreads, ROWS * COLS>(s, tile_e);
        __syncthreads();
        ix_compute<TY, SPEC>(reinterpret_cast<const int2*>(s), g.out, g.nx, g.ny, g.periodic, x0, y0, g.itaps,
                             w, tile_e);
      }
    } else {
      if constexpr (sd.xform) xform_tile<T>(s, ROWS * COLS);
      spec_compute<T, TY, SPEC>(s, g.out, g.nx, g.ny, g.periodic, x0, y0, g.taps);
    }
  }
}

template <typename T, int TY, int SPEC, int MODE>
int launch_group(const GroupTable<T>& tab, cudaStream_t st) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  const size_t smem = tile_smem_bytes<T>(sd.L, sd.R, sd.T, sd.B, TY, false);
  auto kern = k_stencil2d_group<T, TY, SPEC, MODE>;
  static int per_sm = 0;  // resident CTAs per SM of this instantiation (set on first use)
  if (per_sm == 0) {
    CS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int occ = 0;
    CS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem));
    per_sm = occ > 0 ? occ : -1;
  }
  if (per_sm < 0) return set_error(CS_EUNSUPPORTED, "grouped stencil kernel does not fit on an SM");
  const int grid = static_cast<int>(std::min<int64_t>(tab.total_tiles, static_cast<int64_t>(num_sms()) * per_sm));
  kern<<<static_cast<unsigned>(grid), kThreads, smem, st>>>(tab);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

template <typename T, int TY, int MODE>
int dispatch_group(int variant, const GroupTable<T>& tab, cudaStream_t st) {
  switch (variant) {
#define CS_GR_CASE(I) \
  case I: return launch_group<T, TY, I, MODE>(tab, st);
    CS_GR_CASE(0) CS_GR_CASE(1) CS_GR_CASE(2) CS_GR_CASE(3) CS_GR_CASE(4)
    CS_GR_CASE(5) CS_GR_CASE(6) CS_GR_CASE(7) CS_GR_CASE(8) CS_GR_CASE(9)
    CS_GR_CASE(10) CS_GR_CASE(11) CS_GR_CASE(12) CS_GR_CASE(13)
#undef CS_GR_CASE
    default: return set_error(CS_EINVAL, "internal: unknown stencil variant %d", variant);
  }
}

// Launches up to kMaxGroup plans (same dtype, specialised variant and tile rows) as one grid.
// FP64 plans take the digit path when every plan in the group allows it (integer weight ratios,
// FP64 mode auto), else native FP64.
template <typename T>
int launch_group_t(const Stencil2DConfig* const* cfgs, const void* const* ins, void* const* outs,
                   int count, cudaStream_t st) {
  GroupTable<T> tab;
  memset(&tab, 0, sizeof tab);
  const int variant = cfgs[0]->variant, TY = cfgs[0]->tile_rows;
  const SpecDesc& sd = kSpecs[variant];
  const int nt = (sd.L + sd.R + 1) * (sd.T + sd.B + 1);
  bool digits = sizeof(T) == 8 && !sd.xform;
  int tiles = 0;
  for (int j = 0; j < count; ++j) {
    const Stencil2DConfig* c = cfgs[j];
    GroupJob<T>& g = tab.job[tab.count];
    if (c->nx == 0 || c->ny == 0) continue;
    g.in = static_cast<const T*>(ins[j]);
    g.out = static_cast<T*>(outs[j]);
    g.nx = c->nx;
    g.ny = c->ny;
    g.tiles_x = static_cast<int>((c->nx + tile_x<T>() - 1) / tile_x<T>());
    const int64_t ty = (c->ny + TY - 1) / TY;
    if (static_cast<int64_t>(tiles) + g.tiles_x * ty > 0x7fffffff)
      return set_error(CS_EINVAL, "grouped launch too large");
    g.tile_begin = tiles;
    tiles += static_cast<int>(g.tiles_x * ty);
    g.periodic = c->bc == CS_BC_PERIODIC;
    g.vec_ok = (c->nx % Vec<T>::n == 0) && (reinterpret_cast<uintptr_t>(ins[j]) % 16 == 0);
    for (int i = 0; i < 32; ++i) g.taps.w[i] = i < nt ? static_cast<T>(c->weights[i]) : T(0);
    digits = digits && c->ix_ok && c->fp64_mode == CS_FP64_AUTO;
    for (int i = 0; i < 32; ++i) g.itaps.n[i] = static_cast<int8_t>(i < nt && c->ix_ok ? c->ix_n[i] : 0);
    g.itaps.c = ixd::ixi_round51(c->ix_c);
    g.itaps.c15 = -1.5 * g.itaps.c;
    if (c->ix_ok) {
      g.itaps.inv_hi = static_cast<float>(1.0 / c->ix_c);
      g.itaps.inv_lo = static_cast<float>(1.0 / c->ix_c - static_cast<double>(g.itaps.inv_hi));
    }
    ++tab.count;
  }
  tab.total_tiles = tiles;
  if (tab.count == 0) return CS_OK;
  if constexpr (sizeof(T) == 8) {
    if (digits)
      return TY == 32 ? dispatch_group<T, 32, 1>(variant, tab, st) : dispatch_group<T, 64, 1>(variant, tab, st);
  }
  return TY == 32 ? dispatch_group<T, 32, 0>(variant, tab, st) : dispatch_group<T, 64, 0>(variant, tab, st);
}

// ---- double-float evaluation of FP64-storage stencils ---------------------------------------
// GB300 issues FP64 at 2 DFMA/clk/SM against ~128 FP32 ops/clk/SM, so FP64-storage sweeps are
// evaluated in double-float arithmetic (Dekker 1971: a value is an unevaluated sum hi + lo of
// two floats) on the FP32 pipes.  Every element is split with integer operations (the
// f64 -> f32 conversion instruction itself runs on the FP64 pipe); each tap adds the exact
// product of the split weight and value (FMA error term) into an error-free TwoSum
// accumulator; the result is hi + lo rounded once to FP64.  The error is below ~2^-46 of
// sum|w| * max|in|.  A tile whose values leave the safe exponent range (or whose largest value
// is tiny) is evaluated in native FP64 instead, so results stay correct for every input.

struct DDTaps { float hi[32], lo[32]; };

constexpr int kDDMinExp = 1023 - 70;   // smallest biased exponent split on the fast path
constexpr int kDDMaxExp = 1023 + 60;   // first biased exponent that is not
constexpr int kDDTileExp = 1023 - 30;  // a tile's largest value must reach 2^-30 (or be 0)

// x = hi + lo: hi is x truncated to 24 significant bits, lo the remainder rounded to 24 bits.
// Returns false outside the fast exponent range; ebias = biased exponent (0 for +-0).
__device__ __forceinline__ bool dd_split(double x, float& hi, float& lo, int& ebias) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const uint32_t top = static_cast<uint32_t>(b >> 32);
  const uint32_t sign = top & 0x80000000u;
  const int e = static_cast<int>((top >> 20) & 0x7ffu);
  if ((b << 1) == 0) {
    hi = __uint_as_float(sign);
    lo = 0.0f;
    ebias = 0;
    return true;
  }
  ebias = e;
  if (e < kDDMinExp || e >= kDDMaxExp) return false;
  const uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  hi = __uint_as_float(sign | (static_cast<uint32_t>(e - 1023 + 127) << 23) | static_cast<uint32_t>(mant >> 29));
  const uint32_t rem = static_cast<uint32_t>(mant & 0x1FFFFFFFu);            // 29 low bits
  const float scale = __uint_as_float(static_cast<uint32_t>(e - 1075 + 127) << 23);  // 2^(e-1075)
  lo = __fmul_rn(__uint2float_rn(rem), scale);
  lo = __uint_as_float(__float_as_uint(lo) | sign);
  return true;
}

// Exact float -> double on the integer pipe.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) {
    if ((b & 0x7fffffffu) == 0u) return __longlong_as_double(static_cast<long long>(b & 0x80000000u) << 32);
    return static_cast<double>(f);  // subnormal / inf / nan: rare
  }
  const uint64_t d = (static_cast<uint64_t>(b & 0x80000000u) << 32) | (static_cast<uint64_t>(e + 896u) << 52) |
                     (static_cast<uint64_t>(b & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(d));
}

// Splits the N staged FP64 values (N even) in place: each 16-byte pair of values becomes
// (hi0, hi1, lo0, lo1).  Returns, uniformly over the block, whether the double-float path
// applies to the tile; when it does not, the tile still holds the FP64 values.
template <int N>
__device__ __forceinline__ bool dd_split_tile(double* s, int* s_red) {
  constexpr int NPAIR = N / 2, PER = (NPAIR + kThreads - 1) / kThreads;
  const double2* q = reinterpret_cast<const double2*>(s);
  float4 v[PER];
  bool ok = true;
  int maxe = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int k = static_cast<int>(threadIdx.x) + j * kThreads;
    if (k < NPAIR) {
      const double2 d = q[k];
      float h0, l0, h1, l1;
      int e0, e1;
      ok = dd_split(d.x, h0, l0, e0) && ok;
      ok = dd_split(d.y, h1, l1, e1) && ok;
      maxe = max(maxe, max(e0, e1));
      v[j] = make_float4(h0, h1, l0, l1);
    }
  }
  maxe = __reduce_max_sync(0xffffffffu, maxe);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = maxe;
  const bool all_ok = __syncthreads_and(ok);
  int tile_e = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) tile_e = max(tile_e, s_red[w]);
  const bool use = all_ok && (tile_e == 0 || tile_e >= kDDTileExp);
  if (use) {
    float4* o = reinterpret_cast<float4*>(s);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int k = static_cast<int>(threadIdx.x) + j * kThreads;
      if (k < NPAIR) o[k] = v[j];
    }
    __syncthreads();
  }
  return use;
}

// Double-float stencil of two adjacent tile columns per thread, "push" form (each staged row
// adds its taps to the up to H output rows it feeds, in the order (row, column) of the taps, as
// a one-output-at-a-time evaluation would).  A row is read as 16-byte (hi, hi, lo, lo) column
// pairs; taps at an odd column offset take their pair from two neighbouring loads.
template <int TY, int SPEC>
__device__ __forceinline__ void dd_compute(const float4* sp, double* __restrict__ out, int64_t nx,
                                           int64_t ny, int periodic, int64_t x0, int64_t y0,
                                           const DDTaps& taps) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int L = sd.L, R = sd.R, TT = sd.T, BB = sd.B;
  constexpr int V = Vec<double>::n;
  constexpr int TX = tile_x<double>();
  static_assert(TX == 64, "one warp spans the tile's 64 columns");
  constexpr int LA = (L + V - 1) / V * V, RA = (R + V - 1) / V * V;
  constexpr int COLS = LA + TX + RA, CP = COLS / 2;
  constexpr int W = L + R + 1, H = TT + BB + 1;
  constexpr int WY = kThreads / 32, RW = TY / WY;
  constexpr int S0 = LA - L, X = S0 & 1, NP = (W + 1 + X + 1) / 2;  // pairs read per row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = 2 * lane;
  const int r0 = warp * RW;
  const int64_t gx = x0 + c;
  const bool ok0 = gx < nx && (periodic || (gx >= L && gx < nx - R));
  const bool ok1 = gx + 1 < nx && (periodic || (gx + 1 >= L && gx + 1 < nx - R));
  const bool both = ok0 && ok1 && (reinterpret_cast<uintptr_t>(out) & 15u) == 0 && (nx & 1) == 0;
  const int64_t gy0 = y0 + r0;
  const int64_t ylo = periodic ? 0 : TT, yhi = periodic ? ny : ny - BB;
  auto rows_below = [](int64_t d) { return static_cast<int>(d < 0 ? 0 : (d > RW ? RW : d)); };
  const int klo = rows_below(ylo - gy0);
  const int khi = (ok0 || ok1) ? rows_below(yhi - gy0) : 0;
  double* op = out + gy0 * nx + gx;
  const float4* a = sp + (S0 - X + c) / 2;
  float2 sh[H], sl[H];
#pragma unroll
  for (int q = 0; q < H; ++q) sh[q] = sl[q] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int i = 0; i < RW + H - 1; ++i) {
    float4 P[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      bool used = false;
#pragma unroll
      for (int q = 0; q < H; ++q)
#pragma unroll
        for (int p = 0; p < W; ++p) {
          const int e = X + p;
          used |= ((e >> 1) == k || ((e + 1) >> 1) == k) && ((sd.mask >> (q * W + p)) & 1u) &&
                  (i - q >= 0) && (i - q < RW);
        }
      if (used) P[k] = a[(r0 + i) * CP + k];
    }
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const int o = i - q;
      if (o < 0 || o >= RW) continue;
#pragma unroll
      for (int p = 0; p < W; ++p)
        if ((sd.mask >> (q * W + p)) & 1u) {
          const int e = X + p;
          float2 xh, xl;
          if ((e & 1) == 0) {
            xh = make_float2(P[e >> 1].x, P[e >> 1].y);
            xl = make_float2(P[e >> 1].z, P[e >> 1].w);
          } else {
            xh = make_float2(P[e >> 1].y, P[(e >> 1) + 1].x);
            xl = make_float2(P[e >> 1].w, P[(e >> 1) + 1].z);
          }
          dd_mac2(sh[o % H], sl[o % H], taps.hi[q * W + p], taps.lo[q * W + p], xh, xl);
        }
    }
    const int done = i - (H - 1);
    if (done >= 0) {
      float2& h = sh[done % H];
      float2& l = sl[done % H];
      if constexpr (sd.epi) {
        const float4 u = sp[(r0 + done + TT) * CP + (LA + c) / 2];  // centre values
        dd_add_cubic_minus2(h, l, make_float2(u.x, u.y), make_float2(u.z, u.w));
      }
      // hi converts on the FP64 pipe (idle enough here), lo on the integer pipe
      const double val0 = static_cast<double>(h.x) + f2d_exact(l.x);
      const double val1 = static_cast<double>(h.y) + f2d_exact(l.y);
      h = l = make_float2(0.0f, 0.0f);
      if (done >= klo && done < khi) {
        if (both) {
          *reinterpret_cast<double2*>(op) = make_double2(val0, val1);
        } else {
          if (ok0) op[0] = val0;
          if (ok1) op[1] = val1;
        }
      }
      op += nx;
    }
  }
}

template <int TY, int SPEC>
__global__ void __launch_bounds__(kThreads)
    k_stencil2d_dd(const double* __restrict__ in, double* __restrict__ out, int64_t nx, int64_t ny,
                   int periodic, int vec_ok, Taps<double> taps, DDTaps dtaps, int ty0) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int V = Vec<double>::n;
  constexpr int TX = tile_x<double>();
  constexpr int LA = (sd.L + V - 1) / V * V, RA = (sd.R + V - 1) / V * V;
  constexpr int COLS = LA + TX + RA, ROWS = TY + sd.T + sd.B;
  static_assert(COLS % 2 == 0, "the split takes values in pairs");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s = reinterpret_cast<double*>(smem_raw);
  __shared__ int s_red[kThreads / 32];
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * TX;
  const int64_t y0 = (static_cast<int64_t>(blockIdx.y) + ty0) * TY;
  load_tile_ct<double, ROWS, COLS>(s, in, nx, ny, periodic != 0, vec_ok != 0, x0, y0, sd.T, LA);
  if constexpr (sd.xform) xform_tile<double>(s, ROWS * COLS);
  if (dd_split_tile<ROWS * COLS>(s, s_red))
    dd_compute<TY, SPEC>(reinterpret_cast<const float4*>(s), out, nx, ny, periodic, x0, y0, dtaps);
  else
    spec_compute<double, TY, SPEC>(s, out, nx, ny, periodic, x0, y0, taps);
}

template <int TY, int SPEC>
int launch_dd(const double* in, double* out, int64_t nx, int64_t ny, int periodic, int vec_ok,
              const Taps<double>& taps, const DDTaps& dtaps, cudaStream_t st) {
  constexpr SpecDesc sd = kSpecs[SPEC];
  const size_t smem = tile_smem_bytes<double>(sd.L, sd.R, sd.T, sd.B, TY, false);
  auto kern = k_stencil2d_dd<TY, SPEC>;
  static bool attr_set = false;
  if (!attr_set) {
    CS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    attr_set = true;
  }
  int ty0, nty;
  window_tiles(TY, ny, &ty0, &nty);
  if (nty == 0) return CS_OK;
  dim3 grid(static_cast<unsigned>((nx + tile_x<double>() - 1) / tile_x<double>()), static_cast<unsigned>(nty));
  kern<<<grid, kThreads, smem, st>>>(in, out, nx, ny, periodic, vec_ok, taps, dtaps, ty0);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

template <int TY>
int dispatch_dd(int variant, const double* in, double* out, int64_t nx, int64_t ny, int periodic,
                int vec_ok, const Taps<double>& taps, const DDTaps& dtaps, cudaStream_t st) {
  switch (variant) {
#define CS_DD_CASE(I) \
  case I: return launch_dd<TY, I>(in, out, nx, ny, periodic, vec_ok, taps, dtaps, st);
    CS_DD_CASE(0) CS_DD_CASE(1) CS_DD_CASE(2) CS_DD_CASE(3) CS_DD_CASE(4)
    CS_DD_CASE(5) CS_DD_CASE(6) CS_DD_CASE(7) CS_DD_CASE(8) CS_DD_CASE(9)
    CS_DD_CASE(10) CS_DD_CASE(11) CS_DD_CASE(12) CS_DD_CASE(13)
#undef CS_DD_CASE
    default: return set_error(CS_EINVAL, "internal: unknown stencil variant %d", variant);
  }
}

// ---- TMA-pipelined persistent sweep ------------------------------------------------------------
// Persistent CTAs walk their tiles (t = blockIdx.x, blockIdx.x + gridDim.x, ...) through a
// two-stage shared-memory ring.  One thread fills a stage with a single 2D tensor-memory-access
// copy (cp.async.bulk.tensor) of the tile plus halo, completed on the stage's mbarrier, so the
// next tile's load overlaps the current tile's compute.  The copy zero-fills cells outside the
// grid; for periodic boundaries the threads of an edge tile then overwrite those cells with the
// wrapped values.  MODE 0 computes in the storage type, MODE 1 is the exact digit path and
// MODE 2 the double-float path of FP64 storage (each with its native-FP64 tile fallback).
// Every mbarrier wait is bounded.  When one runs out (in any thread: the decision is made
// block-wide), thread 0 adds 1 to the plan's *status counter and waits, bounded again, for the
// copies this CTA still has in flight; then the CTA returns with its remaining tiles unwritten.
// The host reads the counter with cs_plan_check.  stall_from (a test hook, INT_MAX when off)
// makes the CTA issue no copy for its tiles from that index on, so the wait for such a tile runs
// out with nothing in flight; those waits use the short kStallWaitLimit.

constexpr int kStages = 2;
constexpr long long kWaitLimit = 1ll << 22;
constexpr long long kStallWaitLimit = 1ll << 10;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Periodic halo of an edge tile: cells outside the grid get their wrapped values.  Only the
// out-of-range strips are visited (whole rows above / below the grid, then the columns left /
// right of it); a grid at least as large as the tile wraps with one compare-and-add.
template <typename T, int COLS, int ROWS>
__device__ __forceinline__ void fixup_periodic(T* s, const T* __restrict__ in, int64_t nx, int64_t ny,
                                               int64_t gx0, int64_t gy0) {
  const bool one_wrap = nx >= COLS && ny >= ROWS;
  auto wx = [&](int64_t g) { return one_wrap ? (g < 0 ? g + nx : (g >= nx ? g - nx : g)) : wrap_idx(g, nx); };
  auto wy = [&](int64_t g) { return one_wrap ? (g < 0 ? g + ny : (g >= ny ? g - ny : g)) : wrap_idx(g, ny); };
  auto clamp = [](int64_t v, int64_t lo, int64_t hi) { return static_cast<int>(v < lo ? lo : (v > hi ? hi : v)); };
  const int r_lo = clamp(-gy0, 0, ROWS);            // rows [0, r_lo) lie above the grid
  const int r_hi = clamp(ny - gy0, r_lo, ROWS);     // rows [r_hi, ROWS) lie below it
  const int c_lo = clamp(-gx0, 0, COLS);
  const int c_hi = clamp(nx - gx0, c_lo, COLS);
  const int out_rows = r_lo + (ROWS - r_hi);
  for (int idx = threadIdx.x; idx < out_rows * COLS; idx += kThreads) {  // whole rows
    const int rr = idx / COLS, c = idx - rr * COLS;
    const int r = rr < r_lo ? rr : r_hi + (rr - r_lo);
    s[r * COLS + c] = in[wy(gy0 + r) * nx + wx(gx0 + c)];
  }
  const int side = c_lo + (COLS - c_hi);
  const int mid_rows = r_hi - r_lo;
  for (int idx = threadIdx.x; idx < mid_rows * side; idx += kThreads) {  // side columns
    const int rr = idx / side, cc = idx - rr * side;
    const int r = r_lo + rr;
    const int c = cc < c_lo ? cc : c_hi + (cc - c_lo);
    s[r * COLS + c] = in[(gy0 + r) * nx + wx(gx0 + c)];
  }
}

template <int MODE, typename T, int SPEC>
struct TmaGeom {
  static constexpr SpecDesc sd = kSpecs[SPEC];
  static constexpr int TY = 64;
  static constexpr int V = Vec<T>::n;
  static constexpr int TX = tile_x<T>();
  static constexpr int LA = (sd.L + V - 1) / V * V, RA = (sd.R + V - 1) / V * V;
  static constexpr int COLS = LA + TX + RA, ROWS = TY + sd.T + sd.B;
  static constexpr int SE = ROWS * COLS;
  static constexpr size_t STAGE_BYTES = (SE * sizeof(T) + 127) / 128 * 128;
  static constexpr size_t EXTRA_BYTES = 0;
  static constexpr size_t SMEM = kStages * STAGE_BYTES + EXTRA_BYTES;
};

template <int MODE, typename T, int SPEC>
__global__ void __launch_bounds__(kThreads)
    k_stencil2d_tma(const __grid_constant__ CUtensorMap tmap, const T* __restrict__ in,
                    T* __restrict__ out, int64_t nx, int64_t ny, int periodic, int tiles_x,
                    int tiles, int ty0, Taps<T> taps, IxTaps itaps, DDTaps dtaps, int* status,
                    int stall_from) {
  using G = TmaGeom<MODE, T, SPEC>;
  constexpr SpecDesc sd = kSpecs[SPEC];
  constexpr int TY = G::TY, TX = G::TX, COLS = G::COLS, ROWS = G::ROWS, SE = G::SE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[kStages];
  __shared__ __align__(16) int s_wmax[kThreads / 32];
  const int tid = threadIdx.x;
  if (blockIdx.x >= tiles) return;
  const int my_tiles = (tiles - 1 - static_cast<int>(blockIdx.x)) / static_cast<int>(gridDim.x) + 1;
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(&mbar[st], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int i, int st) {
    const int t = static_cast<int>(blockIdx.x) + i * static_cast<int>(gridDim.x);
    const int bx = t % tiles_x, by = t / tiles_x + ty0;
    fence_proxy_async();  // order this stage's generic-proxy writes before the async copy
    mbar_expect_tx(&mbar[st], static_cast<uint32_t>(SE * sizeof(T)));
    tma_load_2d(smem_raw + st * G::STAGE_BYTES, &tmap, bx * TX - G::LA, by * TY - sd.T, &mbar[st]);
  };
  if (tid == 0)
    for (int st = 0; st < kStages && st < my_tiles && st < stall_from; ++st) issue(st, st);

  for (int i = 0; i < my_tiles; ++i) {
    const int st = i % kStages;
    const bool ok = mbar_wait_bounded(&mbar[st], static_cast<uint32_t>((i / kStages) & 1),
                                      i < stall_from ? kWaitLimit : kStallWaitLimit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicAdd(status, 1);
        // the copies issued into this CTA's stages (tiles i .. i + kStages - 1) land before it leaves
        for (int j = i; j < i + kStages && j < my_tiles && j < stall_from; ++j)
          mbar_wait_bounded(&mbar[j % kStages], static_cast<uint32_t>((j / kStages) & 1), kWaitLimit);
      }
      return;
    }
    T* s = reinterpret_cast<T*>(smem_raw + st * G::STAGE_BYTES);
    const int t = static_cast<int>(blockIdx.x) + i * static_cast<int>(gridDim.x);
    const int64_t x0 = static_cast<int64_t>(t % tiles_x) * TX;
    const int64_t y0 = static_cast<int64_t>(t / tiles_x + ty0) * TY;
    const int64_t gx0 = x0 - G::LA, gy0 = y0 - sd.T;
    if (periodic && (gx0 < 0 || gx0 + COLS > nx || gy0 < 0 || gy0 + ROWS > ny)) {
      fixup_periodic<T, COLS, ROWS>(s, in, nx, ny, gx0, gy0);
      __syncthreads();
    }
    if constexpr (MODE == 0) {
      if constexpr (sd.xform) xform_tile<T>(s, SE);
      spec_compute<T, TY, SPEC>(s, out, nx, ny, periodic, x0, y0, taps);
    } else if constexpr (MODE == 1) {
      static_assert(COLS % 2 == 0, "digit passes take values in pairs");
      const uint32_t mhi = ixd::ix_tile_max_hi<kThreads, SE>(reinterpret_cast<const double*>(s), reinterpret_cast<unsigned*>(s_wmax));
      const int tile_e = static_cast<int>(mhi >> 20);
      uint32_t w[4];
      if (!ixi_consts(itaps.c, itaps.c15, tile_e, w) || (sd.epi && !ixf_tile_ok(tile_e, itaps.c))) {
        spec_compute<double, TY, SPEC>(s, out, nx, ny, periodic, x0, y0, taps);
      } else {
        ixd::ixi_split_tile<kThreads, SE>(s, tile_e);
        __syncthreads();
        ix_compute<TY, SPEC>(reinterpret_cast<const int2*>(s), out, nx, ny, periodic, x0, y0, itaps, w, tile_e);
      }
    } else {
      static_assert(COLS % 2 == 0, "the split takes values in pairs");
      if constexpr (sd.xform) xform_tile<double>(s, SE);
      if (dd_split_tile<SE>(s, s_wmax))
        dd_compute<TY, SPEC>(reinterpret_cast<const float4*>(s), out, nx, ny, periodic, x0, y0, dtaps);
      else
        spec_compute<double, TY, SPEC>(s, out, nx, ny, periodic, x0, y0, taps);
    }
    __syncthreads();  // every thread is done with stage st
    if (tid == 0 && i + kStages < my_tiles && i + kStages < stall_from) issue(i + kStages, st);
  }
}

template <int MODE, typename T, int SPEC>
int launch_tma(const CUtensorMap& map, const T* in, T* out, int64_t nx, int64_t ny, int periodic,
               const Taps<T>& taps, const IxTaps& it, const DDTaps& dt, int* status, int stall_from,
               cudaStream_t st) {
  using G = TmaGeom<MODE, T, SPEC>;
  auto kern = k_stencil2d_tma<MODE, T, SPEC>;
  static int per_sm = 0;  // resident CTAs per SM for this instantiation (set on first use)
  if (per_sm == 0) {
    CS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(G::SMEM)));
    int occ = 0;
    CS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, G::SMEM));
    per_sm = occ > 0 ? occ : -1;
  }
  if (per_sm < 0) return set_error(CS_EUNSUPPORTED, "TMA stencil kernel does not fit on an SM");
  int ty0, nty;
  window_tiles(G::TY, ny, &ty0, &nty);
  const int64_t tiles_x = (nx + G::TX - 1) / G::TX;
  const int64_t tiles = tiles_x * nty;
  if (tiles == 0) return CS_OK;
  if (tiles > 0x7fffffff) return set_error(CS_EINVAL, "grid too large for the TMA sweep");
  const int64_t grid = std::min<int64_t>(tiles, static_cast<int64_t>(num_sms()) * per_sm);
  kern<<<static_cast<unsigned>(grid), kThreads, G::SMEM, st>>>(map, in, out, nx, ny, periodic,
                                                               static_cast<int>(tiles_x), static_cast<int>(tiles),
                                                               ty0, taps, it, dt, status, stall_from);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

template <int MODE, typename T>
int dispatch_tma(int variant, const CUtensorMap& map, const T* in, T* out, int64_t nx, int64_t ny,
                 int periodic, const Taps<T>& taps, const IxTaps& it, const DDTaps& dt, int* status,
                 int stall_from, cudaStream_t st) {
  switch (variant) {
#define CS_TMA_CASE(I)                                                                          \
  case I:                                                                                       \
    if constexpr (MODE == 1 && kSpecs[I].xform)                                                 \
      return set_error(CS_EINVAL, "internal: no digit kernel for variant %d", I);               \
    else                                                                                        \
      return launch_tma<MODE, T, I>(map, in, out, nx, ny, periodic, taps, it, dt, status, stall_from, st);
    CS_TMA_CASE(0) CS_TMA_CASE(1) CS_TMA_CASE(2) CS_TMA_CASE(3) CS_TMA_CASE(4)
    CS_TMA_CASE(5) CS_TMA_CASE(6) CS_TMA_CASE(7) CS_TMA_CASE(8) CS_TMA_CASE(9)
    CS_TMA_CASE(10) CS_TMA_CASE(11) CS_TMA_CASE(12) CS_TMA_CASE(13)
#undef CS_TMA_CASE
    default: return set_error(CS_EINVAL, "internal: unknown stencil variant %d", variant);
  }
}

// Any extents up to CS_MAX_EXTENT; weights staged in shared memory after the tile.
template <typename T, int TY>
__global__ void __launch_bounds__(kThreads)
    k_stencil2d_generic(const T* __restrict__ in, T* __restrict__ out, int64_t nx, int64_t ny,
                        int periodic, int vec_ok, int L, int R, int TT, int BB,
                        const T* __restrict__ wts, int xform, int epi, int ty0) {
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
  const int64_t y0 = (static_cast<int64_t>(blockIdx.y) + ty0) * TY;
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
  int ty0, nty;
  window_tiles(TY, ny, &ty0, &nty);
  if (nty == 0) return CS_OK;
  dim3 grid(static_cast<unsigned>((nx + tile_x<T>() - 1) / tile_x<T>()), static_cast<unsigned>(nty));
  kern<<<grid, kThreads, smem, st>>>(in, out, nx, ny, periodic, vec_ok, taps, ty0);
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
  int ty0, nty;
  window_tiles(TY, cfg->ny, &ty0, &nty);
  if (nty == 0) return CS_OK;
  dim3 grid(static_cast<unsigned>((cfg->nx + tile_x<T>() - 1) / tile_x<T>()), static_cast<unsigned>(nty));
  kern<<<grid, kThreads, smem, st>>>(in, out, cfg->nx, cfg->ny, periodic, vec_ok, cfg->left,
                                     cfg->right, cfg->top, cfg->bottom, d_w, xform, epi, ty0);
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

int make_tensor_map(const Stencil2DConfig* cfg, const void* in, int elem_bytes, int cols, int rows);

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
    if (cfg->use_tma && vec_ok && cfg->nx < (int64_t(1) << 31) && cfg->ny < (int64_t(1) << 31)) {
      constexpr int V = Vec<T>::n;
      const int LA = (sd.L + V - 1) / V * V, RA = (sd.R + V - 1) / V * V;
      const int cols = LA + tile_x<T>() + RA, rows = 64 + sd.T + sd.B;
      if (cfg->tmap_in != vin) {
        int rc = make_tensor_map(cfg, vin, sizeof(T), cols, rows);
        if (rc != CS_OK) return rc;
      }
      int* status = cfg->d_status;
      if (!status) return set_error(CS_EINVAL, "internal: plan without a status word");
      const int stall = cfg->stall_from < 0 ? 0x7fffffff : cfg->stall_from;
      IxTaps it{};
      DDTaps dt{};
      int mode = 0;
      if constexpr (sizeof(T) == 8) {
        if (cfg->fp64_mode == CS_FP64_AUTO && cfg->ix_ok) {
          mode = 1;
          for (int i = 0; i < 32; ++i) it.n[i] = static_cast<int8_t>(i < nt ? cfg->ix_n[i] : 0);
          it.c = ixd::ixi_round51(cfg->ix_c);
          it.c15 = -1.5 * it.c;
          it.inv_hi = static_cast<float>(1.0 / cfg->ix_c);
          it.inv_lo = static_cast<float>(1.0 / cfg->ix_c - static_cast<double>(it.inv_hi));
        } else if (cfg->fp64_mode == CS_FP64_AUTO && cfg->dd_ok) {
          mode = 2;
          for (int i = 0; i < 32; ++i) {
            const double w = i < nt ? cfg->weights[i] : 0.0;
            dt.hi[i] = static_cast<float>(w);
            dt.lo[i] = static_cast<float>(w - static_cast<double>(dt.hi[i]));
          }
        }
      }
      if constexpr (sizeof(T) == 8) {
        if (mode == 1)
          return dispatch_tma<1, T>(cfg->variant, cfg->tmap, in, out, cfg->nx, cfg->ny, periodic, taps, it, dt, status, stall, st);
        if (mode == 2)
          return dispatch_tma<2, T>(cfg->variant, cfg->tmap, in, out, cfg->nx, cfg->ny, periodic, taps, it, dt, status, stall, st);
      }
      return dispatch_tma<0, T>(cfg->variant, cfg->tmap, in, out, cfg->nx, cfg->ny, periodic, taps, it, dt, status, stall, st);
    }
    if constexpr (sizeof(T) == 8) {
      if (cfg->ix_ok && cfg->fp64_mode == CS_FP64_AUTO) {
        IxTaps it;
        for (int i = 0; i < 32; ++i) it.n[i] = static_cast<int8_t>(i < nt ? cfg->ix_n[i] : 0);
        it.c = ixd::ixi_round51(cfg->ix_c);
        it.c15 = -1.5 * it.c;
        it.inv_hi = static_cast<float>(1.0 / cfg->ix_c);
        it.inv_lo = static_cast<float>(1.0 / cfg->ix_c - static_cast<double>(it.inv_hi));
        if (cfg->tile_rows == 32)
          return dispatch_ix<32>(cfg->variant, in, out, cfg->nx, cfg->ny, periodic, vec_ok, taps, it, cfg, st);
        return dispatch_ix<64>(cfg->variant, in, out, cfg->nx, cfg->ny, periodic, vec_ok, taps, it, cfg, st);
      }
      if (cfg->dd_ok && cfg->fp64_mode == CS_FP64_AUTO) {
        DDTaps dt;
        for (int i = 0; i < 32; ++i) {
          const double w = i < nt ? cfg->weights[i] : 0.0;
          dt.hi[i] = static_cast<float>(w);
          dt.lo[i] = static_cast<float>(w - static_cast<double>(dt.hi[i]));
        }
        if (cfg->tile_rows == 32)
          return dispatch_dd<32>(cfg->variant, in, out, cfg->nx, cfg->ny, periodic, vec_ok, taps, dt, st);
        return dispatch_dd<64>(cfg->variant, in, out, cfg->nx, cfg->ny, periodic, vec_ok, taps, dt, st);
      }
    }
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
