// Exact digit evaluation of integer-weight sums of FP64 values on the integer pipe (GB300 issues
// FP64 at 1/64 of the FP32 rate).  For weights w_k = c * n_k with integers n_k, sum |n_k| <= 64:
// every staged value of a tile is cut into two 24-bit integer digits on a grid fixed by the
// tile's largest exponent, x = (d0 2^24 + d1) 2^(G-48) + r with 0 <= |r| < 2^(G-48), r of the sign
// of x (|x| is truncated on the grid), d0 signed and 0 <= d1 < 2^24, so each digit sum
// S_i = sum_k n_k d_{k,i} is exact in int32.
// T = S0 2^24 + S1 is then rounded to a multiple of 2^4 (ties to even) and scaled by c * 2^(G-48)
// with one FP64 FMA: the result is within (2^-47 + 2^-44 / sum|n| + 2^-50) of sum|w| * (largest
// value of the tile), the last term for c's rounding to 51 bits and the FMA's own rounding.  With
// sum |n_k| <= 8, 28-bit digits keep 56 bits and round to 2^(G-49).  The per-tile constants come
// from c's bits by integer exponent arithmetic, and nothing converts between integers and floating point (on GB300 those conversions share the FP64
// pipe).  Used by the 2D stencil sweep and by the Laplacians of the Cahn-Hilliard right-hand side.
#pragma once

#include <stdint.h>
#include <string.h>

namespace cs {
namespace ixd {

constexpr int kMinExp = 1023 - 900;  // smallest biased exponent of a tile's largest value
constexpr int kMaxExp = 1023 + 900;  // largest one
constexpr int kIDigitBits = 24;
constexpr int kIFracBits = 2 * kIDigitBits;  // bits kept below the tile's top 2^G

// Largest high word (sign cleared) of the N staged FP64 values (N even, 16-byte aligned): its top
// bits are the largest biased exponent, and it is >= 0x7ff00000 exactly when the tile holds an
// inf or a nan.  Every thread of the block (NT threads) gets the result; s_red holds NT / 32 words
// (16-byte aligned).  The trip count is fixed at compile time: every thread takes the same number
// of full rounds, and one guarded round covers the remainder.
template <int NT, int N>
__device__ __forceinline__ uint32_t ix_tile_max_hi(const double* s, unsigned* s_red) {
  static_assert(N % 2 == 0 && NT % 128 == 0, "pairs of values; whole uint4 reads of s_red");
  constexpr int P = N / 2, FULL = P / NT, REM = P % NT;
  const uint4* q = reinterpret_cast<const uint4*>(s);
  uint32_t m = 0u;
#pragma unroll
  for (int it = 0; it < FULL; ++it) {
    const uint4 v = q[threadIdx.x + it * NT];
    m = __vimax3_u32(m, v.y & 0x7fffffffu, v.w & 0x7fffffffu);
  }
  if (REM != 0 && static_cast<int>(threadIdx.x) < REM) {
    const uint4 v = q[threadIdx.x + FULL * NT];
    m = __vimax3_u32(m, v.y & 0x7fffffffu, v.w & 0x7fffffffu);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
  __syncthreads();
  const uint4* r4 = reinterpret_cast<const uint4*>(s_red);
  uint32_t r = 0u;
#pragma unroll
  for (int w = 0; w < NT / 128; ++w) {
    const uint4 v = r4[w];
    r = __vimax3_u32(r, v.x, v.y);
    r = __vimax3_u32(r, v.z, v.w);
  }
  return r;
}

// Digit widths: DB = 24 (the default) keeps 48 bits below 2^G and serves sum |n_k| <= 64;
// DB = 28 keeps 56 bits (every bit of a value within a factor 8 of the tile's largest) and serves
// sum |n_k| <= 8 with the positive n_k summing to at most 7 (S1 <= 7 (2^28 - 1) leaves room for the
// rounding's carry in int32), e.g. the 5-point Laplacian.  RS is the rounding shift of the
// combination, chosen so that |T'| < 2^51: |T| < (sum |n_k|) 2^(2 DB).
template <int DB> struct Digits;
template <> struct Digits<24> { static constexpr int kFrac = 48, kRound = 4, kMaxSum = 64; };
template <> struct Digits<28> { static constexpr int kFrac = 56, kRound = 8, kMaxSum = 8; };

// The common weight scale c as the combination uses it: rounded to 51 significant bits (at most two
// units in c's last place, 2^-51 relative; the weights' own FP64 rounding is 2^-53), so that
// 1.5 c is exact too.
__host__ __device__ inline double ixi_round51(double c) {
  unsigned long long b;
  memcpy(&b, &c, sizeof b);
  b = (b + 2ull) & ~3ull;  // nearest on the two lowest significand bits; a carry moves the exponent
  memcpy(&c, &b, sizeof b);
  return c;
}

// Logical right shift of a 64-bit value; PTX clamps shift amounts above 64 to 64 (result 0), so
// no range test is needed.
__device__ __forceinline__ unsigned long long ixi_shr64(unsigned long long v, int sh) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(sh));
  return r;
}

// Digits of x on the grid whose top is 2^G, G = tile_e - 1022, F = 2 DB: A = floor(|x| / 2^(G-F))
// = M >> (tile_e - e + 53 - F) for the 53-bit significand M of x (biased exponent e <= tile_e;
// for F > 53, M << (F - 53) >> (tile_e - e)), then As = sgn(x) A in two's complement and
// d0 = As >> DB (arithmetic), d1 = As mod 2^DB, so d0 2^DB + d1 = As exactly.  Branch-free.
// Zeros and subnormals: a digit tile has tile_e >= kMinExp, so the shift is >= 64 and A is 0; an
// all-zero tile (tile_e 0) is scaled by 0.
template <int DB = 24>
__device__ __forceinline__ int2 ixi_split(double x, int tile_e) {
  constexpr int F = Digits<DB>::kFrac;
  const uint32_t hi = static_cast<uint32_t>(__double2hiint(x));
  const uint32_t lo = static_cast<uint32_t>(__double2loint(x));
  const int e = static_cast<int>((hi >> 20) & 0x7ffu);
  const unsigned long long M = (static_cast<unsigned long long>((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
  unsigned long long A;
  if constexpr (F <= 53)
    A = ixi_shr64(M, tile_e - e + 53 - F);
  else
    A = ixi_shr64(M << (F - 53), tile_e - e);
  const long long sgn = static_cast<long long>(static_cast<int>(hi) >> 31);  // 0 or -1
  const long long As = (static_cast<long long>(A) ^ sgn) - sgn;
  return make_int2(static_cast<int>(As >> DB), static_cast<int>(As & ((1ll << DB) - 1)));
}

// T * 2^-RS * (2^RS scale) for T = S0 2^DB + S1, with one FP64 instruction:
// T' = S0 2^(DB-RS) + round(S1 / 2^RS) = round(T / 2^RS) (ties to even) is exact apart from the
// last term.  q = qa 2^(DB-RS) + qb (default 0) is an integer added in the same units (the user
// function's cubic term), split so that it joins the two 32-bit parts before the one 64-bit
// multiply-add; |T' + q| < 2^51.  V = T' + q + 2^51 lies in [0, 2^52), so D = 2^52 + V is the bit
// pattern of 2^52 plus V, and fma(D, 2^RS scale, -1.5 2^(52+RS) scale) = (V - 2^51) 2^RS scale is
// rounded once; both constants are exact (ixi_consts, with c rounded to 51 bits).  w holds their
// words.
template <int DB = 24>
__device__ __forceinline__ double ixi_combine(int S0, int S1, const uint32_t (&w)[4], int qa = 0, int qb = 0) {
  constexpr int RS = Digits<DB>::kRound;
  // round(S1 / 2^RS) with ties to even: rounding half up would bias every output by half a unit
  // of 2^-RS on average, and a conserved sum (the Cahn-Hilliard mass) would drift by that much
  const int r = (S1 + ((1 << (RS - 1)) - 1) + ((S1 >> RS) & 1)) >> RS;
  const long long V = static_cast<long long>(S0 + qa) * (1ll << (DB - RS)) + static_cast<long long>(r + qb) +
                      (1ll << 51);
  const double D = __longlong_as_double(static_cast<long long>(0x4330000000000000ull) + V);
  const double sc = __hiloint2double(static_cast<int>(w[0]), static_cast<int>(w[1]));
  const double cs = __hiloint2double(static_cast<int>(w[2]), static_cast<int>(w[3]));
  return __fma_rn(D, sc, cs);
}

// The combination's constants for a tile, scale = c 2^(G-F): w = the words of 2^RS scale and of
// -1.5 2^(52+RS) scale, made by adding to the exponent fields of c and of c15 = -1.5 c (c rounded
// to 51 bits by ixi_round51, so c15 is exact).  Returns false (the tile then takes native FP64)
// when c is zero or not normal, when the tile's largest value is outside [2^-900, 2^900], or when
// either constant would leave the normal range; an all-zero tile (tile_e 0) gets zero constants,
// so its outputs are 0.
template <int DB = 24>
__device__ __forceinline__ bool ixi_consts(double c, double c15, int tile_e, uint32_t (&w)[4]) {
  constexpr int k1 = Digits<DB>::kRound - Digits<DB>::kFrac, k2 = k1 + 52;
  w[0] = w[1] = w[2] = w[3] = 0u;
  if (tile_e == 0) return true;
  const uint32_t chi = static_cast<uint32_t>(__double2hiint(c)), clo = static_cast<uint32_t>(__double2loint(c));
  const uint32_t dhi = static_cast<uint32_t>(__double2hiint(c15)), dlo = static_cast<uint32_t>(__double2loint(c15));
  const int ec = static_cast<int>((chi >> 20) & 0x7ffu), ed = static_cast<int>((dhi >> 20) & 0x7ffu);
  const int G = tile_e - 1022;
  if (tile_e < kMinExp || tile_e > kMaxExp || ec == 0 || ec == 0x7ff) return false;
  if (ec + G + k1 < 1 || ed + G + k2 > 2046) return false;
  w[0] = chi + (static_cast<uint32_t>(G + k1) << 20);
  w[1] = clo;
  w[2] = dhi + (static_cast<uint32_t>(G + k2) << 20);
  w[3] = dlo;
  return true;
}

// Replaces the N staged FP64 values (N even, 16-byte aligned) by their integer digits (d0, d1)
// in the values' own 8-byte slots.  Each of the NT threads converts two values at a time, in a
// compile-time number of rounds (one guarded round for the remainder).
template <int NT, int N, int DB = 24>
__device__ __forceinline__ void ixi_split_tile(double* s, int tile_e) {
  static_assert(N % 2 == 0, "values in pairs");
  constexpr int P = N / 2, FULL = P / NT, REM = P % NT;
  const double2* q = reinterpret_cast<const double2*>(s);
  int4* qi = reinterpret_cast<int4*>(s);
  auto pair = [&](int k) {
    const double2 v = q[k];
    const int2 a = ixi_split<DB>(v.x, tile_e);
    const int2 b = ixi_split<DB>(v.y, tile_e);
    qi[k] = make_int4(a.x, a.y, b.x, b.y);
  };
#pragma unroll 4
  for (int it = 0; it < FULL; ++it) pair(threadIdx.x + it * NT);
  if (REM != 0 && static_cast<int>(threadIdx.x) < REM) pair(threadIdx.x + FULL * NT);
}

}  // namespace ixd
}  // namespace cs
