// Exact digit evaluation of integer-weight sums of FP64 values on the FP32 / integer pipes
// (GB300 issues FP64 at 1/64 of the FP32 rate).  For weights w_k = c * n_k with integers n_k,
// sum |n_k| <= 64: every staged value of a tile is cut into three signed 18-bit digits on a grid
// fixed by the tile's largest exponent, x = sum_i d_i 2^(G - 18(i+1)) (bits below 2^(G-54)
// dropped), so each digit sum S_i = sum_k n_k d_{k,i} is an integer below 2^24 and exact in FP32.
// T = S0 2^36 + S1 2^18 + S2 is then rounded to a multiple of 2^8 and scaled by c * 2^(G-54) with
// one FP64 FMA: the result is within 2^-45 / sum|n| of sum|w| * (largest value of the tile).
// Used by the 2D stencil sweep and by the Laplacians of the Cahn-Hilliard right-hand side.
#pragma once

#include <stdint.h>

namespace cs {
namespace ixd {

constexpr int kDigitBits = 18;
constexpr int kMinExp = 1023 - 900;  // smallest biased exponent of a tile's largest value
constexpr int kMaxExp = 1023 + 900;  // largest one


// Digits of x on the tile grid whose top is 2^G with G = tile_e - 1022 (tile_e = largest biased
// exponent in the tile): A = |x| / 2^(G-54) truncated (54 bits), d0 = A >> 36, d1 and d2 the next
// 18-bit groups, each carrying the sign of x.  Works on the two 32-bit words of x with funnel
// shifts: A = (M << 1) >> (tile_e - e), M the 53-bit significand.
__device__ __forceinline__ void ix_split(double x, int tile_e, float& d0, float& d1, float& d2) {
  const uint32_t hi = static_cast<uint32_t>(__double2hiint(x));
  const uint32_t lo = static_cast<uint32_t>(__double2loint(x));
  const int e = static_cast<int>((hi >> 20) & 0x7ffu);
  // (M << 1) as two words, 22 + 32 bits.  Zeros and subnormals (e == 0) need no special case: a
  // digit tile has tile_e >= kMinExp, so t >= 54 and every digit is 0, and an all-zero tile
  // (tile_e == 0) is scaled by 0.
  const uint32_t mh = __funnelshift_l(lo, (hi & 0xFFFFFu) | 0x100000u, 1);
  const uint32_t ml = lo << 1;
  const int t = tile_e - e;  // >= 0
  uint32_t ah, al;
  if (t < 32) {
    al = __funnelshift_r(ml, mh, t);
    ah = mh >> t;
  } else {
    al = t < 54 ? (mh >> (t - 32)) : 0u;
    ah = 0u;
  }
  // a digit a < 2^18 becomes +-(2^23 + a) by setting the mantissa bits of +-2^23 (exact), and
  // subtracting +-2^23 leaves +-a
  const uint32_t K = 0x4B000000u | (hi & 0x80000000u);
  const float k = __uint_as_float(K);
  d0 = __fsub_rn(__uint_as_float((ah >> 4) | K), k);
  d1 = __fsub_rn(__uint_as_float((__funnelshift_r(al, ah, 18) & 0x3FFFFu) | K), k);
  d2 = __fsub_rn(__uint_as_float((al & 0x3FFFFu) | K), k);
}

// T * scale for T = S0 * 2^36 + S1 * 2^18 + S2 (the digit sums are integers below 2^24 in
// magnitude, so |T| < sum|n| * 2^54 <= 2^60) with one FP64 instruction and no int64 -> FP64
// conversion (GB300 issues about 2 FP64 instructions per clock per SM, the digit kernel's bound):
// T' = round(T / 2^8) = S0 * 2^28 + S1 * 2^10 + round(S2 / 2^8) is exact apart from the last
// term, |T'| <= 2^52, so D = 2^52 + |T'| is assembled by an integer add to the bit pattern of
// 2^52, and fma(D, +-2^8 scale, -+2^60 scale) = T' * 2^8 * scale is rounded once.  sc and cs are
// the two words of 2^8 * scale and of -2^60 * scale (exact power-of-two multiples); the sign of
// T flips both.  Error before the final rounding: at most 2^7 units of 2^(G-54) * |c|.
__device__ __forceinline__ double ix_combine(float S0, float S1, float S2, uint32_t sc_hi, uint32_t sc_lo,
                                            uint32_t cs_hi, uint32_t cs_lo) {
  const long long Tp = (static_cast<long long>(__float2int_rn(S0)) << 28) +
                       (static_cast<long long>(__float2int_rn(S1)) << 10) +
                       static_cast<long long>(__float2int_rn(S2 * 0x1p-8f));
  const uint32_t sgn = static_cast<uint32_t>(static_cast<unsigned long long>(Tp) >> 63) << 31;
  const unsigned long long A = sgn ? 0ull - static_cast<unsigned long long>(Tp) : static_cast<unsigned long long>(Tp);
  const double D = __longlong_as_double(static_cast<long long>(0x4330000000000000ull + A));
  const double sc = __hiloint2double(static_cast<int>(sc_hi ^ sgn), static_cast<int>(sc_lo));
  const double cs = __hiloint2double(static_cast<int>(cs_hi ^ sgn), static_cast<int>(cs_lo));
  return __fma_rn(D, sc, cs);
}

// A tile takes the digit path when its largest value lies in [2^-900, 2^900] and its scale
// c * 2^(G-54) keeps 2^8 scale normal and 2^60 scale finite; an all-zero tile (tile_e 0, scale 0)
// gives zeros.  Every other tile (inf / nan, out-of-range values) is evaluated in native FP64.
__device__ __forceinline__ bool ix_tile_ok(int tile_e, double scale) {
  if (tile_e == 0) return true;
  const double a = fabs(scale);
  return tile_e >= kMinExp && tile_e <= kMaxExp && a >= 0x1p-1000 && a < 0x1p960;
}

// Largest high word (sign cleared) of the n staged FP64 values (n even, 16-byte aligned): its top
// bits are the largest biased exponent, and it is >= 0x7ff00000 exactly when the tile holds an
// inf or a nan.  Every thread of the block (NT threads) gets the result; s_red holds NT / 32 words.
template <int NT>
__device__ __forceinline__ uint32_t ix_tile_max_hi(const double* s, int n, unsigned* s_red) {
  const uint4* q = reinterpret_cast<const uint4*>(s);
  uint32_t m = 0u;
  for (int k = threadIdx.x; k < n / 2; k += NT) {
    const uint4 v = q[k];
    m = __vimax3_u32(m, v.y & 0x7fffffffu, v.w & 0x7fffffffu);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
  __syncthreads();
  uint32_t r = 0u;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) r = max(r, s_red[w]);
  return r;
}

// Replaces the n staged FP64 values by their digits: (d0, d1) pairs over the values' own slots,
// d2 in s2 (8-byte aligned).  Each of the NT threads converts and overwrites two values at a time.
template <int NT>
__device__ __forceinline__ void ix_split_tile(double* s, float* s2, int n, int tile_e) {
  const double2* q = reinterpret_cast<const double2*>(s);
  float4* q01 = reinterpret_cast<float4*>(s);
  float2* q2 = reinterpret_cast<float2*>(s2);
  for (int k = threadIdx.x; k < n / 2; k += NT) {
    const double2 v = q[k];
    float a0, a1, a2, b0, b1, b2;
    ix_split(v.x, tile_e, a0, a1, a2);
    ix_split(v.y, tile_e, b0, b1, b2);
    q01[k] = make_float4(a0, a1, b0, b1);
    q2[k] = make_float2(a2, b2);
  }
}

}  // namespace ixd
}  // namespace cs
