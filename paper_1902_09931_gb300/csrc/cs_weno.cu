// Periodic XY WENO advection (Sec. 4.2, "Advection"): the variant of the periodic XY stencil
// whose inputs are the field C and the velocities u, v, and whose per-point computation is a
// WENO solver instead of a weighted sum.  The output is the advection term
//     a = u C_x + v C_y,
// each derivative the fifth-order WENO approximation for Hamilton-Jacobi equations (Osher &
// Fedkiw, "Level Set Methods and Dynamic Implicit Surfaces", Sec. 3.4 -- the reference the paper
// gives for its solver), upwinded: the left-biased approximation where the velocity component is
// positive, the right-biased one elsewhere.  The stencil is 3 points each way along x and along
// y, no corners (the paper's variant drops the corner loads too).
//
// Tiles: 64 x 32 outputs per CTA of 256 threads; C (with a 3-point periodic halo) staged in
// shared memory by the 2D stencil's tile loader; u and v read once per point from global memory.
// A thread owns one column and walks 8 consecutive rows, keeping its 7-point y window in
// registers.  FP32 fields: FP32 arithmetic.  FP64 fields: the differences and the output in FP64,
// the weights in exact integer and double-float arithmetic (below), with the all-FP64 formula
// kept for points outside that path's range.
//
// The weights.  With v1..v5 the five one-sided differences, candidates phi_k, smoothness
// indicators S_k and q_k = (S_k + eps)^2, the WENO value is
//     sum_k g_k phi_k / q_k  /  sum_k g_k / q_k  =  sum_k g_k phi_k P_k / sum_k g_k P_k,
// P_1 = q_2 q_3, P_2 = q_1 q_3, P_3 = q_1 q_2, g = (0.1, 0.6, 0.3): one division.  The differences
// are first scaled by the power of two 2^-E that brings max|v_k| into [1, 2) (exact), so every
// q_k lies in [1e-12, 2e4] and no product under- or overflows; the scheme is invariant under that
// scaling except for eps's constant floor, which is scaled with it (1e-99 h^2 2^-2E).  Where the
// floor is at least 1e19 times every S_k, the weights equal g to rounding and the linear
// combination sum_k g_k phi_k is taken directly (this covers all-zero and tiny differences).

#include <cmath>
#include <cstring>

#include "cs_internal.h"
#include "cs_stencil2d_kernels.cuh"

namespace cs {
namespace {

constexpr int kWThreads = 256;
constexpr int kWTX = 64;                        // columns per tile
constexpr int kWTY = 32;                        // rows per tile
constexpr int kWHalo = 3;                       // stencil reach along x and y
constexpr int kWGroups = kWThreads / kWTX;      // row groups
constexpr int kWRows = kWTY / kWGroups;         // rows per thread
constexpr int kWLA = 4;                         // left halo, rounded up to 16 bytes in both types
constexpr int kWCols = kWLA + kWTX + kWLA;
constexpr int kWTileRows = kWTY + 2 * kWHalo;

__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }

// The WENO value from the scaled differences w1..w5 (max |w_k| in [1, 2)), eps = 1e-6 max w^2 + fl.
template <typename T>
__device__ __forceinline__ T weno_scaled(T w1, T w2, T w3, T w4, T w5, T mw, T fl) {
  const T phi1 = fma_(T(1.0 / 3.0), w1, fma_(T(-7.0 / 6.0), w2, T(11.0 / 6.0) * w3));
  const T phi2 = fma_(T(-1.0 / 6.0), w2, fma_(T(5.0 / 6.0), w3, T(1.0 / 3.0) * w4));
  const T phi3 = fma_(T(1.0 / 3.0), w3, fma_(T(5.0 / 6.0), w4, T(-1.0 / 6.0) * w5));
  const T a1 = fma_(T(-2), w2, w1) + w3, b1 = fma_(T(-4), w2, w1) + T(3) * w3;
  const T a2 = fma_(T(-2), w3, w2) + w4, b2 = w2 - w4;
  const T a3 = fma_(T(-2), w4, w3) + w5, b3 = fma_(T(3), w3, fma_(T(-4), w4, w5));
  const T s1 = fma_(T(13.0 / 12.0) * a1, a1, T(0.25) * b1 * b1);
  const T s2 = fma_(T(13.0 / 12.0) * a2, a2, T(0.25) * b2 * b2);
  const T s3 = fma_(T(13.0 / 12.0) * a3, a3, T(0.25) * b3 * b3);
  const T eps = fma_(T(1e-6), mw * mw, fl);
  const T t1 = s1 + eps, t2 = s2 + eps, t3 = s3 + eps;
  const T q1 = t1 * t1, q2 = t2 * t2, q3 = t3 * t3;
  const T p1 = T(0.1) * (q2 * q3), p2 = T(0.6) * (q1 * q3), p3 = T(0.3) * (q1 * q2);
  const T num = fma_(p1, phi1, fma_(p2, phi2, p3 * phi3));
  const T den = p1 + p2 + p3;
  // FP32: the fast division (2 ulp; den lies in [1e-24, 3e8], inside its range) -- FP32 storage
  // is held to 1e-5
  if constexpr (sizeof(T) == 4) return __fdividef(num, den);
  else return num / den;
}

// sum_k g_k phi_k: the optimal-weight (linear) combination, (2 v1 - 13 v2 + 47 v3 + 27 v4 - 3 v5) / 60.
template <typename T>
__device__ __forceinline__ T weno_linear(T v1, T v2, T v3, T v4, T v5) {
  const T phi1 = fma_(T(1.0 / 3.0), v1, fma_(T(-7.0 / 6.0), v2, T(11.0 / 6.0) * v3));
  const T phi2 = fma_(T(-1.0 / 6.0), v2, fma_(T(5.0 / 6.0), v3, T(1.0 / 3.0) * v4));
  const T phi3 = fma_(T(1.0 / 3.0), v3, fma_(T(5.0 / 6.0), v4, T(-1.0 / 6.0) * v5));
  return fma_(T(0.1), phi1, fma_(T(0.6), phi2, T(0.3) * phi3));
}

// WENO value of unscaled differences v1..v5 (in units of C; the caller divides by h), with
// floor_h2 = 1e-99 h^2 the eps floor in those units: all in FP64.
__device__ __noinline__ double weno5_fp64(double v1, double v2, double v3, double v4, double v5, double floor_h2) {
  const double m = fmax(fmax(fmax(fabs(v1), fabs(v2)), fmax(fabs(v3), fabs(v4))), fabs(v5));
  const int e = static_cast<int>(__double_as_longlong(m) >> 52);  // biased exponent of max |v|
  // e < 600: max|v| < 2^-423 and the floor (>= 1e-99 * 1e-120 for h >= 1e-60) outweighs every
  // S_k by far more than 1e19; e > 2045: inf / nan or next to overflow (kept linear)
  if (e >= 600 && e <= 2045) {
    const double sc = __longlong_as_double(static_cast<long long>(2046 - e) << 52);  // 2^(1023 - e)
    const double fl = floor_h2 * sc * sc;
    if (fl < 1e19) {
      const double r = weno_scaled<double>(v1 * sc, v2 * sc, v3 * sc, v4 * sc, v5 * sc, m * sc, fl);
      return r * __longlong_as_double(static_cast<long long>(e) << 52);  // * 2^(e - 1023)
    }
  }
  return weno_linear<double>(v1, v2, v3, v4, v5);
}

// ---- FP64 storage, mixed precision ------------------------------------------------------------
// GB300 issues FP64 at 1/64 of the FP32 rate, so only the steps that need FP64's 53 bits stay on
// the FP64 pipe: the one-sided differences and the second differences a_k, b_k of the smoothness
// indicators, where the cancellation happens (the indicators amplify an input error by ~200 in
// the weights when S ~ eps).  Every other step runs in double-float arithmetic (a value as an
// unevaluated pair of floats, error-free products and sums; ~2^-46 relative per operation) on the
// FP32 pipe: the indicators S' = 12 S = 13 a^2 + 3 b^2, the candidates Phi' = 6 phi, eps' = 12 eps,
// (S' + eps')^2, the products with weights 1 : 6 : 3 (the common factors 12^2, 6 and 0.1 cancel in
// the ratio) and the division.  The error stays below ~1e-13 of max|v|.

struct dd { float hi, lo; };
__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dd fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_add(dd x, dd y) {
  const dd s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dd dd_neg(dd x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dd dd_mulf(dd x, float c) {  // c a small integer
  const float p = __fmul_rn(x.hi, c);
  return fast_two_sum(p, __fmaf_rn(x.lo, c, __fmaf_rn(x.hi, c, -p)));
}
__device__ __forceinline__ dd dd_sqr(dd x) {
  const float p = __fmul_rn(x.hi, x.hi);
  return fast_two_sum(p, __fmaf_rn(__fmul_rn(2.0f, x.hi), x.lo, __fmaf_rn(x.hi, x.hi, -p)));
}

// v * 2^(1023 - e) as a float pair, exactly up to the last 6 of v's 52 mantissa bits (relative
// error <= 2^-46), by integer operations only; |v| 2^(1023 - e) < 2^-100 (negligible beside the
// largest difference, >= 1) gives zero.
__device__ __forceinline__ dd split_scaled(double v, int e) {
  const uint32_t hw = static_cast<uint32_t>(__double2hiint(v)), lw = static_cast<uint32_t>(__double2loint(v));
  const int k = static_cast<int>((hw >> 20) & 0x7ffu) - e;  // exponent of the scaled value
  if (((hw >> 20) & 0x7ffu) == 0u || k < -100) return {0.0f, 0.0f};
  const uint32_t sign = hw & 0x80000000u;
  const float hi = __uint_as_float(sign | (static_cast<uint32_t>(k + 127) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  float lo = 0.0f;
  if (k >= -80) {  // next 23 mantissa bits, scaled by 2^(k - 46) (a normal float)
    const float r = __fsub_rn(__uint_as_float(0x4b000000u | ((lw & 0x1fffffffu) >> 6)), 8388608.0f);
    lo = __uint_as_float(__float_as_uint(__fmul_rn(r, __uint_as_float(static_cast<uint32_t>(k + 81) << 23))) | sign);
  }
  return {hi, lo};
}

// ---- exact second differences on the integer pipe ----
// v * 2^(1082 - e) truncated to an integer (|v| < 2^(e - 1022) gives |I| < 2^60, so the indicator
// combinations, at most 8 I in size, stay below 2^63); bits below 2^-60 of max|v| are dropped.
__host__ __device__ __forceinline__ long long fixed_of(unsigned long long bits, int e) {
  const int ev = static_cast<int>((bits >> 52) & 0x7ffu);
  if (ev == 0) return 0;
  const unsigned long long mant = (bits & 0xfffffffffffffull) | (1ull << 52);
  const int sh = ev - e + 7;  // <= 7
  const unsigned long long u = sh >= 0 ? (mant << sh) : (sh > -53 ? (mant >> -sh) : 0ull);
  return (bits >> 63) ? -static_cast<long long>(u) : static_cast<long long>(u);
}

__host__ __device__ __forceinline__ int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll(static_cast<long long>(x));
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ float float_of_bits(unsigned int b) {
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
}

// The integer A (|A| < 2^63) times 2^-59 as a float pair: the leading 24 bits, then the next 24
// (relative error <= 2^-48 of |A|).  A = I-combinations of fixed_of values, so A 2^-59 is the
// combination of the values scaled by 2^(1023 - e).
__host__ __device__ __forceinline__ void dd_of_fixed(long long A, float& hi, float& lo) {
  hi = lo = 0.0f;
  if (A == 0) return;
  const unsigned int sign = A < 0 ? 0x80000000u : 0u;
  unsigned long long U = A < 0 ? static_cast<unsigned long long>(-A) : static_cast<unsigned long long>(A);
  const int p = 63 - clz64(U);  // leading bit
  unsigned long long H = p >= 23 ? (U >> (p - 23)) : (U << (23 - p));
  hi = float_of_bits(sign | (static_cast<unsigned int>(p + 68) << 23) | static_cast<unsigned int>(H & 0x7fffffu));
  if (p <= 23) return;  // no bits left
  const unsigned long long R = U - (H << (p - 23));
  if (R == 0) return;
  const int q = 63 - clz64(R);
  const unsigned long long L = q >= 23 ? (R >> (q - 23)) : (R << (23 - q));
  lo = float_of_bits(sign | (static_cast<unsigned int>(q + 68) << 23) | static_cast<unsigned int>(L & 0x7fffffu));
}

// 12e-6 as a float pair
constexpr float kEps12Hi = 1.2e-5f;
constexpr float kEps12Lo = static_cast<float>(1.2e-5 - static_cast<double>(1.2e-5f));

__device__ __forceinline__ double weno5(double v1, double v2, double v3, double v4, double v5, double floor_h2) {
  // exact max |v|: non-negative doubles order as their bit patterns
  const unsigned long long mask = 0x7fffffffffffffffull;
  unsigned long long mb = static_cast<unsigned long long>(__double_as_longlong(v1)) & mask;
  mb = max(mb, static_cast<unsigned long long>(__double_as_longlong(v2)) & mask);
  mb = max(mb, static_cast<unsigned long long>(__double_as_longlong(v3)) & mask);
  mb = max(mb, static_cast<unsigned long long>(__double_as_longlong(v4)) & mask);
  mb = max(mb, static_cast<unsigned long long>(__double_as_longlong(v5)) & mask);
  const int e = static_cast<int>(mb >> 52);
  // fl = floor_h2 2^(2 (1023 - e)), by exponent arithmetic (floor_h2 is a normal double: h >= 1e-60)
  const unsigned long long fb = static_cast<unsigned long long>(__double_as_longlong(floor_h2));
  const int fe = static_cast<int>(fb >> 52) + 2 * (1023 - e);  // biased exponent of fl
  // fl >= 2^19 (the floor outweighs the indicators), or max|v| outside the scaled range: FP64
  if (e < 600 || e > 2045 || fe >= 1023 + 19) return weno5_fp64(v1, v2, v3, v4, v5, floor_h2);
  const double fl = fe >= 1 ? __longlong_as_double(static_cast<long long>((fb & 0xfffffffffffffull) |
                                                                        (static_cast<unsigned long long>(fe) << 52)))
                            : 0.0;
  // the second differences of the indicators, exactly, in 64-bit integers
  const long long i1 = fixed_of(static_cast<unsigned long long>(__double_as_longlong(v1)), e);
  const long long i2 = fixed_of(static_cast<unsigned long long>(__double_as_longlong(v2)), e);
  const long long i3 = fixed_of(static_cast<unsigned long long>(__double_as_longlong(v3)), e);
  const long long i4 = fixed_of(static_cast<unsigned long long>(__double_as_longlong(v4)), e);
  const long long i5 = fixed_of(static_cast<unsigned long long>(__double_as_longlong(v5)), e);
  // double-float from here, on values scaled by 2^(1023 - e)
  const dd w1 = split_scaled(v1, e), w2 = split_scaled(v2, e), w3 = split_scaled(v3, e);
  const dd w4 = split_scaled(v4, e), w5 = split_scaled(v5, e);
  auto ind = [&](long long a, long long b) {  // 12 S = 13 a^2 + 3 b^2
    dd da, db;
    dd_of_fixed(a, da.hi, da.lo);
    dd_of_fixed(b, db.hi, db.lo);
    return dd_add(dd_mulf(dd_sqr(da), 13.0f), dd_mulf(dd_sqr(db), 3.0f));
  };
  const dd s1 = ind(i1 - 2 * i2 + i3, i1 - 4 * i2 + 3 * i3);
  const dd s2 = ind(i2 - 2 * i3 + i4, i2 - i4);
  const dd s3 = ind(i3 - 2 * i4 + i5, 3 * i3 - 4 * i4 + i5);
  // 6 phi_k
  const dd p1 = dd_add(dd_add({__fmul_rn(2.0f, w1.hi), __fmul_rn(2.0f, w1.lo)}, dd_mulf(w2, -7.0f)), dd_mulf(w3, 11.0f));
  const dd p2 = dd_add(dd_add(dd_neg(w2), dd_mulf(w3, 5.0f)), {__fmul_rn(2.0f, w4.hi), __fmul_rn(2.0f, w4.lo)});
  const dd p3 = dd_add(dd_add({__fmul_rn(2.0f, w3.hi), __fmul_rn(2.0f, w3.lo)}, dd_mulf(w4, 5.0f)), dd_neg(w5));
  // 12 eps = 12e-6 max w^2 + 12 floor
  const dd mw = split_scaled(__longlong_as_double(static_cast<long long>(mb)), e);
  dd eps = dd_mul(dd_sqr(mw), {kEps12Hi, kEps12Lo});
  if (fe >= 1023 - 100) eps = dd_add(eps, dd_mulf(split_scaled(fl, 1023), 12.0f));  // else < 2^-99: below eps's last bit
  const dd q1 = dd_sqr(dd_add(s1, eps)), q2 = dd_sqr(dd_add(s2, eps)), q3 = dd_sqr(dd_add(s3, eps));
  const dd P1 = dd_mul(q2, q3), P2 = dd_mulf(dd_mul(q1, q3), 6.0f), P3 = dd_mulf(dd_mul(q1, q2), 3.0f);
  const dd num = dd_add(dd_add(dd_mul(P1, p1), dd_mul(P2, p2)), dd_mul(P3, p3));
  const dd den = dd_add(dd_add(P1, P2), P3);
  // num / den: one correction step on a correctly rounded reciprocal
  const float rcp = __frcp_rn(den.hi);
  const float y1 = __fmul_rn(num.hi, rcp);
  const dd r = dd_add(num, dd_neg(dd_mulf(den, y1)));
  const dd y = fast_two_sum(y1, __fmul_rn(r.hi, rcp));
  // back to FP64: (hi + lo) * 2^(e - 1023) / 6
  const double sixth = __longlong_as_double(static_cast<long long>(0x3fc5555555555555ull + (static_cast<unsigned long long>(e - 1023) << 52)));
  return (s2d::f2d_exact(y.hi) + s2d::f2d_exact(y.lo)) * sixth;
}

// FP32: the floor (1e-99 h^2, below FP32's range) is left out; it changes eps by a relative
// 1e-99 h^2 / (1e-6 max v^2), i.e. nothing unless the differences are denormal.
__device__ __forceinline__ float weno5(float v1, float v2, float v3, float v4, float v5, float) {
  const float m = fmaxf(fmaxf(fmaxf(fabsf(v1), fabsf(v2)), fmaxf(fabsf(v3), fabsf(v4))), fabsf(v5));
  const int e = static_cast<int>(__float_as_uint(m) >> 23);
  if (e >= 1 && e <= 253) {
    const float sc = __uint_as_float(static_cast<unsigned>(254 - e) << 23);  // 2^(127 - e)
    const float r = weno_scaled<float>(v1 * sc, v2 * sc, v3 * sc, v4 * sc, v5 * sc, m * sc, 0.f);
    return r * __uint_as_float(static_cast<unsigned>(e) << 23);  // * 2^(e - 127)
  }
  return weno_linear<float>(v1, v2, v3, v4, v5);
}

// u > 0 by the bit pattern (integer compare; a nan with the sign bit clear counts as positive,
// which changes nothing: the term is nan either way)
__device__ __forceinline__ bool positive(double u) { return __double_as_longlong(u) > 0; }
__device__ __forceinline__ bool positive(float u) { return __float_as_int(u) > 0; }

// d[k] = C(i + k - 2) - C(i + k - 3), k = 0..5 (the differences at i - 3 .. i + 2); upwind
// selection: left-biased (d0..d4) for a positive velocity, right-biased (d5..d1) otherwise.
template <typename T>
__device__ __forceinline__ T upwind(const T (&d)[6], bool pos, T floor_h2) {
  const T v1 = pos ? d[0] : d[5];
  const T v2 = pos ? d[1] : d[4];
  const T v3 = pos ? d[2] : d[3];
  const T v4 = pos ? d[3] : d[2];
  const T v5 = pos ? d[4] : d[1];
  return weno5(v1, v2, v3, v4, v5, floor_h2);
}

// FP64 storage: at least 4 CTAs per SM (the mixed-precision body then fits 63 registers without
// spilling; measured 2.6 % faster than the compiler's 69 registers and 3 CTAs).
template <typename T>
__global__ void __launch_bounds__(kWThreads, sizeof(T) == 8 ? 4 : 1)
    k_weno_adv(const T* __restrict__ c, const T* __restrict__ u, const T* __restrict__ v, T* __restrict__ out,
               int64_t nx, int64_t ny, int vec_ok, T inv_hx, T inv_hy, T floor_x, T floor_y) {
  __shared__ __align__(16) T s[kWTileRows * kWCols];
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * kWTX;
  const int64_t y0 = static_cast<int64_t>(blockIdx.y) * kWTY;
  s2d::load_tile<T>(s, c, nx, ny, true, vec_ok != 0, x0, y0, kWHalo, kWLA, kWCols, kWTileRows);
  const int tx = threadIdx.x % kWTX;
  const int r0 = (threadIdx.x / kWTX) * kWRows;
  const int64_t gx = x0 + tx;
  if (gx >= nx) return;
  const T* colp = s + tx + kWLA;
  T col[2 * kWHalo + 1];  // C at rows y - 3 .. y + 3 of this column
#pragma unroll
  for (int k = 0; k < 2 * kWHalo + 1; ++k) col[k] = colp[(r0 + k) * kWCols];
  // the row loop stays rolled for FP64 storage: its double-float body is large, and unrolled
  // copies overflow the instruction cache
#pragma unroll(sizeof(T) == 4 ? kWRows : 1)
  for (int r = 0; r < kWRows; ++r) {
    const int64_t gy = y0 + r0 + r;
    if (gy >= ny) break;
    const T* row = colp + (r0 + r + kWHalo) * kWCols;
    T dx[6], dy[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      dx[k] = row[k - 2] - row[k - 3];
      dy[k] = col[k + 1] - col[k];
    }
    const int64_t o = gy * nx + gx;
    const T uu = u[o], vv = v[o];
    const T fx = upwind<T>(dx, positive(uu), floor_x) * inv_hx;
    const T fy = upwind<T>(dy, positive(vv), floor_y) * inv_hy;
    out[o] = fma_(uu, fx, vv * fy);
    if (r + 1 < kWRows) {
#pragma unroll
      for (int k = 0; k < 2 * kWHalo; ++k) col[k] = col[k + 1];
      col[2 * kWHalo] = colp[(r0 + r + 2 * kWHalo + 1) * kWCols];
    }
  }
}

// ---- FP32 storage: two adjacent columns per thread in packed FP32x2 arithmetic -----------------
// The WENO weights of two neighbouring outputs run as one chain of FP32x2 instructions (each lane
// rounds as the scalar form would); the upwind choice, the exponent of max|v| and the division
// stay per lane.  Tiles of 128 x 32 outputs: 64 column pairs x 4 row groups of 8 rows; a row's
// x window (10 values) is read as five 8-byte loads, the y windows roll in registers.
constexpr int kW2TX = 128, kW2Cols = kWLA + kW2TX + kWLA, kW2Groups = kWThreads / (kW2TX / 2);
constexpr int kW2Rows = kWTY / kW2Groups;

__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
// a - b on two lanes as one packed FMA (a packed FMA has no free operand sign)
__device__ __forceinline__ float2 sub2w(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.0f), a); }

// The WENO value of two lanes from their differences w1..w5 (unscaled) and max |w| (mw, with
// 2^-40 <= mw < 2^41), eps = 1e-6 mw^2, in a form with fewer operations than the textbook one
// (the same quantities up to rounding):
//   * with d_k = w_k - w_{k+1}: a_k = d_k - d_{k+1} (the indicators' second differences),
//     b1 = d1 - 3 d2, b2 = d2 + d3, b3 = 3 d3 - d4;
//   * the indicators s_k = (13/12) a_k^2 + (1/4) b_k^2 and eps enter only through their ratios,
//     so S_k = a_k^2 + (3/13) b_k^2 = (12/13) s_k and eps' = (12/13) eps are used;
//   * only the indicator sums are scaled, by sc2 = 2^(2 (127 - e)) (e the biased exponent of mw),
//     so that the fourth powers stay in range: t_k = fma(S_k, sc2, eps' sc2) (a power of two
//     commutes with the roundings);
//   * with q_k = t_k^2 and the weights g = (0.1, 0.6, 0.3) taken as (1, 6, 3), the value is
//     phi_2 + (g1 q2 q3 (phi_1 - phi_2) + g3 q1 q2 (phi_3 - phi_2)) / (g1 q2 q3 + g2 q1 q3 + g3 q1 q2),
//     where phi_1 - phi_2 = (a1 - a2) / 3 and phi_3 - phi_2 = (a2 - a3) / 6 are third differences:
//     phi_2 + (m1 (a1 - a2) + 1.5 m3 (a2 - a3)) / (3 m1 + 18 m2 + 9 m3), m1 = q2 q3, m2 = q1 q3,
//     m3 = q1 q2.
__device__ __forceinline__ float2 weno_scaled2(float2 w1, float2 w2, float2 w3, float2 w4, float2 w5, float2 mw,
                                               float2 sc2) {
  const float2 d1 = sub2w(w1, w2), d2 = sub2w(w2, w3), d3 = sub2w(w3, w4), d4n = sub2w(w5, w4);
  const float2 a1 = sub2w(d1, d2), a2 = sub2w(d2, d3), a3 = __fadd2_rn(d3, d4n);
  const float2 b1 = __ffma2_rn(f2s(-3.0f), d2, d1), b2 = __fadd2_rn(d2, d3), b3 = __ffma2_rn(f2s(3.0f), d3, d4n);
  constexpr float k313 = 3.0f / 13.0f;
  const float2 S1 = __ffma2_rn(a1, a1, __fmul2_rn(__fmul2_rn(f2s(k313), b1), b1));
  const float2 S2 = __ffma2_rn(a2, a2, __fmul2_rn(__fmul2_rn(f2s(k313), b2), b2));
  const float2 S3 = __ffma2_rn(a3, a3, __fmul2_rn(__fmul2_rn(f2s(k313), b3), b3));
  const float2 es = __fmul2_rn(__fmul2_rn(mw, mw), __fmul2_rn(f2s(1e-6f * 12.0f / 13.0f), sc2));
  const float2 t1 = __ffma2_rn(S1, sc2, es), t2 = __ffma2_rn(S2, sc2, es), t3 = __ffma2_rn(S3, sc2, es);
  const float2 q1 = __fmul2_rn(t1, t1), q2 = __fmul2_rn(t2, t2), q3 = __fmul2_rn(t3, t3);
  const float2 m1 = __fmul2_rn(q2, q3), m2 = __fmul2_rn(q1, q3), m3 = __fmul2_rn(q1, q2);
  const float2 den = __ffma2_rn(f2s(18.0f), m2, __ffma2_rn(f2s(9.0f), m3, __fmul2_rn(f2s(3.0f), m1)));
  const float2 num = __ffma2_rn(m1, sub2w(a1, a2), __fmul2_rn(m3, __fmul2_rn(f2s(1.5f), sub2w(a2, a3))));
  const float2 phi2 = __ffma2_rn(f2s(-1.0f / 6.0f), w2, __ffma2_rn(f2s(5.0f / 6.0f), w3, __fmul2_rn(f2s(1.0f / 3.0f), w4)));
  // the fast division's reciprocal (2 ulp; den lies in [1e-24, 2e9], well inside its range) --
  // FP32 storage is held to 1e-5
  return __ffma2_rn(num, make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y)), phi2);
}

// Lanes whose max |w| is zero, denormal or outside [2^-40, 2^41): the scalar form, out of line so
// the unrolled rows of the kernel stay small.
__device__ __noinline__ float2 weno5_pair_slow(float2 v1, float2 v2, float2 v3, float2 v4, float2 v5) {
  return make_float2(weno5(v1.x, v2.x, v3.x, v4.x, v5.x, 0.0f), weno5(v1.y, v2.y, v3.y, v4.y, v5.y, 0.0f));
}

// upwinded WENO derivative (unscaled: the caller divides by h) of two lanes; d[k] the differences
// at k = 0..5 as for upwind(), pos the lanes' velocity signs
__device__ __forceinline__ float2 upwind2(const float2 (&d)[6], bool posx, bool posy) {
  auto pick = [&](int a, int b) { return make_float2(posx ? d[a].x : d[b].x, posy ? d[a].y : d[b].y); };
  const float2 v1 = pick(0, 5), v2 = pick(1, 4), v3 = pick(2, 3), v4 = pick(3, 2), v5 = pick(4, 1);
  auto lane_max = [](float a, float b, float c, float d_, float e) {
    return fmaxf(fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(c), fabsf(d_))), fabsf(e));
  };
  const float mx = lane_max(v1.x, v2.x, v3.x, v4.x, v5.x), my = lane_max(v1.y, v2.y, v3.y, v4.y, v5.y);
  const int ex = static_cast<int>(__float_as_uint(mx) >> 23), ey = static_cast<int>(__float_as_uint(my) >> 23);
  if (ex >= 127 - 40 && ex <= 127 + 40 && ey >= 127 - 40 && ey <= 127 + 40) {
    const float2 sc2 = make_float2(__uint_as_float(static_cast<unsigned>(381 - 2 * ex) << 23),
                                   __uint_as_float(static_cast<unsigned>(381 - 2 * ey) << 23));
    return weno_scaled2(v1, v2, v3, v4, v5, make_float2(mx, my), sc2);
  }
  return weno5_pair_slow(v1, v2, v3, v4, v5);
}

// Dynamic shared memory of k_weno_adv_f32x2: the C tile with its halo, then the u and v tiles.
constexpr size_t kW2Smem = sizeof(float) * (static_cast<size_t>(kWTileRows) * kW2Cols + 2 * kWTY * kW2TX);

__global__ void __launch_bounds__(kWThreads)
    k_weno_adv_f32x2(const float* __restrict__ c, const float* __restrict__ u, const float* __restrict__ v,
                     float* __restrict__ out, int64_t nx, int64_t ny, int vec_ok, int uv_ok, float inv_hx,
                     float inv_hy) {
  extern __shared__ __align__(16) float w2_smem[];
  float* s = w2_smem;                        // C, rows y0 - 3 .. y0 + 34, columns x0 - 4 .. x0 + 131
  float* su = s + kWTileRows * kW2Cols;      // u, rows y0 .. y0 + 31, columns x0 .. x0 + 127
  float* sv = su + kWTY * kW2TX;             // v, likewise
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * kW2TX;
  const int64_t y0 = static_cast<int64_t>(blockIdx.y) * kWTY;
  // u and v of a whole tile are staged with asynchronous 16-byte copies issued before the C tile's,
  // so no row waits on a global load of its own; load_tile's wait covers all of them.  Edge tiles
  // (and unaligned u, v) read u and v per row from global memory.
  const bool staged = uv_ok && x0 + kW2TX <= nx && y0 + kWTY <= ny;
  if (staged) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    static_assert(kW2TX == 4 * 32, "one 16-byte chunk per lane and row");
#pragma unroll
    for (int r = warp; r < kWTY; r += kWThreads / 32) {
      const int64_t g = (y0 + r) * nx + x0 + 4 * lane;
      const unsigned o = static_cast<unsigned>(r * kW2TX + 4 * lane) * static_cast<unsigned>(sizeof(float));
      s2d::cp_async16_s(static_cast<unsigned>(__cvta_generic_to_shared(su)) + o, u + g);
      s2d::cp_async16_s(static_cast<unsigned>(__cvta_generic_to_shared(sv)) + o, v + g);
    }
  }
  s2d::load_tile<float>(s, c, nx, ny, true, vec_ok != 0, x0, y0, kWHalo, kWLA, kW2Cols, kWTileRows);
  const int cx = 2 * (threadIdx.x % (kW2TX / 2));
  const int r0 = (threadIdx.x / (kW2TX / 2)) * kW2Rows;
  const int64_t gx = x0 + cx;
  if (gx >= nx) return;
  const bool two = gx + 1 < nx;
  // both outputs' stores as one 8-byte store where the row start keeps 8-byte alignment
  const bool pair_store = two && (nx % 2 == 0) && (reinterpret_cast<uintptr_t>(out) % 8 == 0) &&
                          (reinterpret_cast<uintptr_t>(u) % 8 == 0) && (reinterpret_cast<uintptr_t>(v) % 8 == 0);
  const float* colp = s + cx + kWLA;  // this thread's first column
  float2 col[2 * kWHalo + 1];         // the two columns at rows y - 3 .. y + 3
#pragma unroll
  for (int k = 0; k < 2 * kWHalo + 1; ++k) col[k] = *reinterpret_cast<const float2*>(colp + (r0 + k) * kW2Cols);
#pragma unroll
  for (int r = 0; r < kW2Rows; ++r) {
    const int64_t gy = y0 + r0 + r;
    if (gy >= ny) break;
    const float* row = colp + (r0 + r + kWHalo) * kW2Cols;
    float w[10];  // columns cx - 4 .. cx + 5 (8-byte aligned pairs)
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float2 t = *reinterpret_cast<const float2*>(row - 4 + 2 * k);
      w[2 * k] = t.x;
      w[2 * k + 1] = t.y;
    }
    float2 dx[6], dy[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {  // C(i + j) is w[4 + j] for lane 0 (column cx), w[5 + j] for lane 1
      dx[k] = make_float2(w[k + 2] - w[k + 1], w[k + 3] - w[k + 2]);
      dy[k] = __ffma2_rn(col[k], f2s(-1.0f), col[k + 1]);
    }
    const int64_t o = gy * nx + gx;
    float2 uu, vv;
    if (staged) {
      uu = *reinterpret_cast<const float2*>(su + (r0 + r) * kW2TX + cx);
      vv = *reinterpret_cast<const float2*>(sv + (r0 + r) * kW2TX + cx);
    } else if (pair_store) {
      uu = *reinterpret_cast<const float2*>(u + o);
      vv = *reinterpret_cast<const float2*>(v + o);
    } else {
      uu = make_float2(u[o], two ? u[o + 1] : 0.0f);
      vv = make_float2(v[o], two ? v[o + 1] : 0.0f);
    }
    const float2 fx = __fmul2_rn(upwind2(dx, positive(uu.x), positive(uu.y)), f2s(inv_hx));
    const float2 fy = __fmul2_rn(upwind2(dy, positive(vv.x), positive(vv.y)), f2s(inv_hy));
    const float2 res = __ffma2_rn(uu, fx, __fmul2_rn(vv, fy));
    if (pair_store) {
      *reinterpret_cast<float2*>(out + o) = res;
    } else {
      out[o] = res.x;
      if (two) out[o + 1] = res.y;
    }
    if (r + 1 < kW2Rows) {
#pragma unroll
      for (int k = 0; k < 2 * kWHalo; ++k) col[k] = col[k + 1];
      col[2 * kWHalo] = *reinterpret_cast<const float2*>(colp + (r0 + r + 2 * kWHalo + 1) * kW2Cols);
    }
  }
}

}  // namespace

int weno_launch(const WenoConfig* cfg, const void* c, const void* u, const void* v, void* out, cudaStream_t st) {
  if (cfg->nx == 0 || cfg->ny == 0) return CS_OK;
  const size_t eb = cfg->dtype == CS_F32 ? 4 : 8;
  const int vec_ok = reinterpret_cast<uintptr_t>(c) % 16 == 0 && (cfg->nx * eb) % 16 == 0;
  const int64_t tx = cfg->dtype == CS_F32 ? kW2TX : kWTX;
  const int64_t gx = (cfg->nx + tx - 1) / tx, gy = (cfg->ny + kWTY - 1) / kWTY;
  if (gx > 0x7fffffff || gy > 65535)
    return set_error(CS_EUNSUPPORTED, "grid %lld x %lld exceeds the WENO launch limits", (long long)cfg->nx, (long long)cfg->ny);
  const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  const double fx = 1e-99 * cfg->hx * cfg->hx, fy = 1e-99 * cfg->hy * cfg->hy;
  if (cfg->dtype == CS_F32) {
    static bool attr_set = false;
    if (!attr_set) {
      CS_CUDA_TRY(cudaFuncSetAttribute(k_weno_adv_f32x2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kW2Smem)));
      attr_set = true;
    }
    const int uv_ok = reinterpret_cast<uintptr_t>(u) % 16 == 0 && reinterpret_cast<uintptr_t>(v) % 16 == 0 &&
                      (cfg->nx * eb) % 16 == 0;
    k_weno_adv_f32x2<<<grid, kWThreads, kW2Smem, st>>>(static_cast<const float*>(c), static_cast<const float*>(u),
                                                       static_cast<const float*>(v), static_cast<float*>(out),
                                                       cfg->nx, cfg->ny, vec_ok, uv_ok,
                                                       static_cast<float>(1.0 / cfg->hx),
                                                       static_cast<float>(1.0 / cfg->hy));
  } else {
    k_weno_adv<double><<<grid, kWThreads, 0, st>>>(static_cast<const double*>(c), static_cast<const double*>(u),
                                                   static_cast<const double*>(v), static_cast<double*>(out), cfg->nx,
                                                   cfg->ny, vec_ok, 1.0 / cfg->hx, 1.0 / cfg->hy, fx, fy);
  }
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

}  // namespace cs
