// Cahn-Hilliard ADI time step with periodic boundaries (Sec. 5.1 of arXiv:1902.09931).
//
//   Cbar = 2 C^n - C^{n-1}
//   RHS  = -(2/3)(C^n - C^{n-1}) - (2/3) D gamma dt lap4(Cbar) + (2/3) D dt lap2(C^3 - C)^n
//   L_x w = RHS,   L_y v = w,   C^{n+1} = Cbar + v,   L = I + a P,  a = (2/3) D gamma dt / h^4
//
// lap2 is the 5-point Laplacian of Eq. 5a and lap4 = dxxxx + 2 dxxyy + dyyyy (Eq. 5b, Fig. 1),
// which on the periodic grid is exactly lap2 applied twice.  The right-hand side is therefore
// evaluated in the factored form
//   Z   = (2/3) D dt / h^2 * N - a * (sum of 4 neighbours of Cbar - 4 Cbar)
//   RHS = -(2/3)(C^n - C^{n-1}) + (sum of 4 neighbours of Z - 4 Z)
// which needs 16 instead of 24 FP64 operations per point (FP64 is the bound on GB300); the two
// Laplacians are exact integer-digit sums, each scaled by one FP64 FMA (the first carrying -a), which
// leaves about 8.6.  FP32 storage evaluates the right-hand side the same way, on exactly widened
// values: its terms reach ~64 a |Cbar| and the solves cancel them back down to |C|, so FP32
// arithmetic there would lose every digit of C at n = 4096 (a = 1.8e5).
//
// Line solves (the paper uses cuPentBatch with the periodic corners treated as in Navon's
// PENT).  Here each periodic line of length n is cut into P chunks of m = n / P points; since
// every chunk block A (m x m pentadiagonal Toeplitz) and every coupling are identical for all
// lines, chunks and steps, the library precomputes once:
//   - the LU factors of A,
//   - the spikes S_L = A^{-1} E_L, S_R = A^{-1} E_R (responses to the two values on each side),
//   - the inverse of the block-circulant 4P x 4P system for the chunk-end values.
// Per sweep, phase 1 solves A g = b on every (line, chunk) independently and records g at the
// chunk ends; phase 2 forms the two end values of each neighbouring chunk from the recorded
// ends (16 P FMAs) and corrects x = g - S_L t_{p-1} - S_R h_{p+1}.  This is exact (up to
// rounding) and gives n * P independent threads instead of n sequential lines.
//
// No-flux boundaries (cs_ch_desc.boundary = CS_CH_NOFLUX): the same step on a cell-centred
// grid whose stencils read ghost cells by even reflection.  Reflection commutes with the
// 5-point Laplacian, so the factored right-hand side holds unchanged -- only the tile loader
// mirrors indices instead of wrapping them.  The line operator is non-cyclic, I + a D4 with the
// reflected fourth difference (first rows (1+2a, -3a, a), (-3a, 1+6a, -4a, a)): the first and
// last chunks of a line get their own LU factors and spikes, the couplings are the same, and the
// chunk-end system is inverted as a dense 4P x 4P matrix (no longer block-circulant; applying it
// still takes 16 P FMAs per chunk).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "cs_digits.cuh"
#include "cs_internal.h"

namespace cs {

struct CHPlan {
  int64_t n;
  int storage;
  double D, gamma, dt, h, a, alpha;
  int P, m;
  void* field[3];
  int iprev, icur, inext;
  int64_t steps;
  double* A;         // n*n scratch (RHS, then w)
  double* B;         // n*n scratch (local solutions g)
  double* bnd;       // 4 * P * n chunk-end values
  double* coef;      // 9 * m line-solve coefficients
  double* K;         // P * 16 block-circulant inverse
  double* partials;  // 2 per RHS block
  double* inv;       // 2 per step (device)
  int64_t inv_cap;
  int rhs_blocks;
  cudaGraphExec_t graph3[3];  // three steps (one buffer rotation) per starting rotation phase
  int graph_kernels;
  double* diag;  // coarsening measures: n/2 twiddles (re, im), 2 n partial sums, 4 results
  int noflux;    // CS_CH_NOFLUX: reflected ghost cells, non-cyclic line solves
};

void drop_graphs(CHPlan* p);

namespace {

constexpr int kTX = 64, kTY = 32, kThreads = 256, kSolveThreads = 32;
constexpr int kU = 8;  // line elements per register batch in the solves

// ---- exact conversions on the integer pipe (f32 <-> f64 conversion runs on the FP64 pipe) ----
__device__ __forceinline__ double widen(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) {
    if ((b & 0x7fffffffu) == 0u) return __longlong_as_double(static_cast<long long>(b & 0x80000000u) << 32);
    return static_cast<double>(f);  // subnormal, inf, nan: rare
  }
  const uint64_t d = (static_cast<uint64_t>(b & 0x80000000u) << 32) |
                     (static_cast<uint64_t>(e + 896u) << 52) |
                     (static_cast<uint64_t>(b & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(d));
}
__device__ __forceinline__ double widen(double d) { return d; }

__device__ __forceinline__ float narrow_rn(double x) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ffu) - 1023 + 127;
  if (e <= 0 || e >= 255) {
    if ((b << 1) == 0) return __uint_as_float(static_cast<uint32_t>(b >> 32));  // +-0
    return __double2float_rn(x);  // subnormal result, overflow, inf, nan: rare
  }
  const uint32_t sign = static_cast<uint32_t>(b >> 32) & 0x80000000u;
  const uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  const uint32_t m23 = static_cast<uint32_t>(mant >> 29);
  const uint32_t rem = static_cast<uint32_t>(mant & 0x1FFFFFFFu);
  uint32_t r = sign | (static_cast<uint32_t>(e) << 23) | m23;
  if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) r += 1u;  // ties to even
  return __uint_as_float(r);
}

// ---- the cubic term of Z on the Laplacian's digit grid ----------------------------------------
// Z = alpha N - a Lap(Cbar), N = u^3 - u (u = C^n).  Lap(Cbar) is an exact digit sum T on the grid
// 2^(G-56) of Cbar's tile, combined as (T' + Q) c 2^(G-48) with T' = round(T / 2^8) and c = -a
// rounded to 51 bits (ixi_combine<28>).  N joins it as the integer Q = round(alpha N / (c 2^(G-48))),
// formed in double-float arithmetic on the FP32 pipe, two points per packed instruction; Z then
// costs the one FP64 FMA of the combination instead of four FP64 operations.  Q is rounded to the
// grid unit c 2^(G-48) that T' already has, so Z's error stays of the size of the Laplacian's own
// rounding.  Used where alpha / |c| <= 2^-6 (the host passes a zero inverse otherwise), which keeps
// the double-float error of Q (<= 2^-46 |alpha N| plus 2^-47 |u| |3u^2 - 1| alpha / |c| in grid
// units) below a tenth of a unit; points outside the ranges below take the FP64 formula.
struct CubicInv { float hi, lo; };  // alpha / c as a float pair, or zero: the FP64 formula

inline CubicInv cubic_inv(double alpha, double c) {
  const double r = alpha / c;
  if (!(std::fabs(r) <= 0.015625) || r == 0.0) return {0.0f, 0.0f};
  const float hi = static_cast<float>(r);
  return {hi, static_cast<float>(r - static_cast<double>(hi))};
}

// (alpha / c) 2^(48 - G) as a float pair, by exponent arithmetic on the host's pair; false when
// the inverse is zero or the scaled pair would leave the normal float range.
__device__ __forceinline__ bool cubic_scaled(CubicInv inv, int tile_e, float& ih, float& il) {
  const int sh = 1070 - tile_e;  // 48 - G, G = tile_e - 1022
  const int eh = static_cast<int>((__float_as_uint(inv.hi) >> 23) & 0xffu) + sh;
  if (inv.hi == 0.0f || eh < 25 || eh > 254) return false;
  ih = __uint_as_float(__float_as_uint(inv.hi) + (static_cast<uint32_t>(sh) << 23));
  const int el = static_cast<int>((__float_as_uint(inv.lo) >> 23) & 0xffu) + sh;
  il = (inv.lo == 0.0f || el < 1) ? 0.0f : __uint_as_float(__float_as_uint(inv.lo) + (static_cast<uint32_t>(sh) << 23));
  return true;
}

// u as the float pair h + l with |u - h - l| < 2^-47 |u|, by integer operations alone: h holds u's
// sign, exponent and leading 24 significand bits, l the next 24 bits.  Valid for biased exponents
// e in [944, 1150]; e = 0 (zero or subnormal) gives h = l = 0.
__device__ __forceinline__ void split_hl(double u, float& h, float& l) {
  const uint32_t hw = static_cast<uint32_t>(__double2hiint(u)), lw = static_cast<uint32_t>(__double2loint(u));
  // hw << 3 | lw >> 29 puts the exponent's low 8 bits over the top 23 significand bits; with the
  // exponent's bit 7 flipped first those 8 bits read e - 896, the float exponent (e in [897, 1150])
  const uint32_t top = __funnelshift_l(lw, hw ^ 0x08000000u, 3);
  const uint32_t hb = (top & 0x7fffffffu) | (hw & 0x80000000u);
  // the next 24 bits as an exact integer times 2^(e - 1070), with u's sign: float exponent e - 943
  const float x = __uint2float_rn((lw >> 5) & 0xffffffu);
  const float sc = __uint_as_float((hb & 0xff800000u) - (47u << 23));
  const bool zero = (hw & 0x7ff00000u) == 0u;
  h = zero ? 0.0f : __uint_as_float(hb);
  l = zero ? 0.0f : __fmul_rn(x, sc);
}

__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.0f), a); }

// Q for two points u = h + l (packed lanes), returned as qa 2^20 + qb, the split ixi_combine<28>
// takes, with qh (|qh| < 2^43 is required; the caller checks it).  Steps, all error-free apart from
// the dropped l^2 and a l terms (2^-48 relative) and the roundings of the small parts:
//   u^2 = A + a2:   nA = -h h rounded, a2 = (h h + nA) + 2 h l
//   u^3 = s3 + b:   ns3 = nA h rounded (= -s3), b = (A h - s3) + A l + a2 h
//   -N = u - u^3 = (ns3 + h) + (l - b) = S + lo (TwoSum of ns3 and h)
//   R = -N (alpha / c) 2^(48 - G) = qh + ql (the product's error by FMA, renormalised by Fast2Sum)
// and Q = -round(R) in two FP32 rounding shifts: 1.5 2^44 takes qh to k 2^21 (k in the low
// mantissa bits), 1.5 2^23 rounds the rest (qh - k 2^21 + ql, |rest| < 2^21) to k2; Q = -(k 2^21 + k2).
__device__ __forceinline__ void cubic_q2(float2 h, float2 l, float ih, float il, int2& qa, int2& qb, float2& qh) {
  const float2 nh = __fmul2_rn(h, f2s(-1.0f)), nl = __fmul2_rn(l, f2s(-1.0f));
  const float2 nA = __fmul2_rn(nh, h);
  const float2 a2 = __ffma2_rn(__fadd2_rn(h, h), l, __ffma2_rn(h, h, nA));
  const float2 ns3 = __fmul2_rn(nA, h);
  float2 b = __ffma2_rn(nA, nh, ns3);
  b = __ffma2_rn(nA, nl, b);
  b = __ffma2_rn(a2, h, b);
  const float2 S = __fadd2_rn(ns3, h);
  const float2 bb = sub2(S, ns3);
  const float2 t = __fadd2_rn(sub2(ns3, sub2(S, bb)), sub2(h, bb));
  const float2 lo = __fadd2_rn(sub2(t, b), l);
  const float2 np = __fmul2_rn(S, f2s(-ih));
  float2 pl = __ffma2_rn(S, f2s(ih), np);
  pl = __ffma2_rn(lo, f2s(ih), pl);
  pl = __ffma2_rn(S, f2s(il), pl);
  qh = sub2(pl, np);
  const float2 ql = sub2(pl, __fadd2_rn(qh, np));
  constexpr float M1 = 26388279066624.0f, M2 = 12582912.0f;  // 1.5 2^44, 1.5 2^23
  const float2 t1 = __fadd2_rn(qh, f2s(M1));
  const float2 rest = __fadd2_rn(sub2(qh, sub2(t1, f2s(M1))), ql);
  const float2 t2 = __fadd2_rn(rest, f2s(M2));
  qa = make_int2(2 * static_cast<int>(__float_as_uint(M1) - __float_as_uint(t1.x)),
                 2 * static_cast<int>(__float_as_uint(M1) - __float_as_uint(t1.y)));
  qb = make_int2(static_cast<int>(__float_as_uint(M2) - __float_as_uint(t2.x)),
                 static_cast<int>(__float_as_uint(M2) - __float_as_uint(t2.y)));
}

// Whether a point may take the digit form: u zero or with biased exponent in [944, tile_e + 1]
// (|u| < 2^(G+1), which bounds the double-float error of Q), |qh| < 2^43 (the rounding shifts'
// range; false for inf and nan), and the Laplacian's high digit sum |S0| <= 2^31 - 2^24, so that
// |T' + Q| < 2^51 as the combination requires.
__device__ __forceinline__ bool cubic_ok(double u, int tile_e, float qh, int s0) {
  const int e = static_cast<int>((static_cast<uint32_t>(__double2hiint(u)) >> 20) & 0x7ffu);
  return (e == 0 || (e >= 944 && e <= tile_e + 1)) && fabsf(qh) < 8796093022208.0f &&
         abs(s0) <= 2147483647 - 16777215;
}

// 2^k as a double (k in the normal range), by its bit pattern
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double(static_cast<long long>(k + 1023) << 52); }

// a 128-bit integer as a double, within 2^-52 of its value: magnitude in two 64-bit halves
__device__ __forceinline__ double i128_to_double(__int128 v) {
  const bool neg = v < 0;
  const unsigned __int128 a = neg ? static_cast<unsigned __int128>(-v) : static_cast<unsigned __int128>(v);
  const double r = fma(__ull2double_rn(static_cast<unsigned long long>(a >> 64)), 18446744073709551616.0,
                       __ull2double_rn(static_cast<unsigned long long>(a)));
  return neg ? -r : r;
}

template <typename T> __device__ __forceinline__ void store_as(T* p, double v);
template <> __device__ __forceinline__ void store_as<double>(double* p, double v) { *p = v; }
template <> __device__ __forceinline__ void store_as<float>(float* p, double v) { *p = narrow_rn(v); }

__device__ __forceinline__ int wrapn(int64_t k, int64_t n) {
  return static_cast<int>(k < 0 ? k + n : (k >= n ? k - n : k));
}
// even reflection about the boundary: -1 -> 0, -2 -> 1, n -> n - 1, n + 1 -> n - 2
__device__ __forceinline__ int mirrorn(int64_t k, int64_t n) {
  return static_cast<int>(k < 0 ? -1 - k : (k >= n ? 2 * n - 1 - k : k));
}
// line-solve chunk type: bit 0 the line's first chunk, bit 1 its last (no-flux tables)
__host__ __device__ __forceinline__ int chunk_type(int p, int P) { return (p == 0 ? 1 : 0) | (p == P - 1 ? 2 : 0); }

// 128-bit shuffle (two 64-bit halves)
__device__ __forceinline__ __int128 shfl_down_i128(__int128 v, int off) {
  const unsigned long long lo = __shfl_down_sync(0xffffffffu, static_cast<unsigned long long>(v), off);
  const long long hi = __shfl_down_sync(0xffffffffu, static_cast<long long>(v >> 64), off);
  return static_cast<__int128>(hi) * (static_cast<__int128>(1) << 64) + static_cast<__int128>(lo);
}

// The block's exact integer invariant sums (mass digits S0, S1; sum U L; sum W^2, see k_ch_rhs),
// reduced in integers over the block (every total stays below 2^127), then converted once to
// FP64 by thread 0: out2 = (sum C, sum energy density) of the block.
__device__ __forceinline__ void block_reduce_int(long long s0, long long s1, __int128 sg, __int128 sw, int G,
                                                 double half_gamma_over_h2, double* out2) {
  __shared__ long long rs[2][kThreads / 32];
  __shared__ __int128 rq[2][kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, off);
    s1 += __shfl_down_sync(0xffffffffu, s1, off);
    sg += shfl_down_i128(sg, off);
    sw += shfl_down_i128(sw, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { rs[0][warp] = s0; rs[1][warp] = s1; rq[0][warp] = sg; rq[1][warp] = sw; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long a = 0, b = 0;
    __int128 g = 0, w = 0;
    for (int k = 0; k < kThreads / 32; ++k) { a += rs[0][k]; b += rs[1][k]; g += rq[0][k]; w += rq[1][k]; }
    out2[0] = fma(static_cast<double>(a), 268435456.0, static_cast<double>(b)) * pow2d(G - 56);
    const double ew = i128_to_double(w) * pow2d(4 * G - 102);
    const double eg = i128_to_double(g) * pow2d(2 * G - 112);
    out2[1] = fma(0.25, ew, -half_gamma_over_h2 * eg);
  }
}

template <typename T>
__device__ __forceinline__ void block_reduce2(double m, double e, double* out2) {
  __shared__ double red[2][kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    m += __shfl_down_sync(0xffffffffu, m, off);
    e += __shfl_down_sync(0xffffffffu, e, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][warp] = m; red[1][warp] = e; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sm = 0.0, se = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) { sm += red[0][w]; se += red[1][w]; }
    out2[0] = sm;
    out2[1] = se;
  }
}

// RHS of the x-sweep and, when partials != nullptr, the per-block FP64 sums of C and of the
// free-energy density of C^n.  rhs == nullptr computes the sums only.  The tile is staged in FP64
// whatever the storage type T (FP32 values widen exactly): the right-hand side carries terms of
// size ~64 a |Cbar| (a = 1.8e5 at n = 4096) that the solves cancel back down to |C|, so it needs
// FP64 precision; evaluated in FP32 it loses all of C's digits at the large grids.  The one
// exception: with FP32 storage Cbar = 2 C^n - C^{n-1} is formed in FP32 (one rounding) exactly as
// the update forms it, then widened.  Both uses of Cbar then agree, so the step is the scheme
// applied to that Cbar, whose rounding reaches C^{n+1} at most undamped (it is of the size of the
// stored result's own rounding); everything after it is FP64.  At least 5 CTAs per SM (the two
// staged tiles' 39 KB of shared memory allow 5): 48 registers, no spills.
template <typename T>
__global__ void __launch_bounds__(kThreads, 5)
    k_ch_rhs(const T* __restrict__ cur, const T* __restrict__ prev, double* __restrict__ rhs, int64_t n,
             double alpha, double a, double half_gamma_over_h2, double* __restrict__ partials, int noflux,
             double am51, CubicInv cinv, int band, T* __restrict__ cbar_out) {
  constexpr int HR = kTY + 4, HC = kTX + 4;  // halo-2 tiles
  constexpr int ZR = kTY + 2, ZC = kTX + 2;  // halo-1 tile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sc = reinterpret_cast<double*>(smem_raw);  // C^n
  double* sb = sc + HR * HC;                         // Cbar, then Z (halo-1 tile) once Cbar is used up
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * kTX;
  const int64_t y0 = static_cast<int64_t>(blockIdx.y) * kTY;
  // band != 0: cur and prev are row bands padded with the 2 rows above and the 2 rows below (the
  // neighbours' rows, exchanged by the caller, or at a no-flux edge of the grid the band's own rows
  // mirrored); output row r of the band is padded row r + 2
  const uintptr_t addr_bits = reinterpret_cast<uintptr_t>(cur) | reinterpret_cast<uintptr_t>(prev) |
                              reinterpret_cast<uintptr_t>(cbar_out);
  const bool inner = x0 >= 2 && x0 + kTX + 2 <= n && (band || (y0 >= 2 && y0 + kTY + 2 <= n)) &&
                     (addr_bits & (2 * sizeof(T) - 1)) == 0;
  if (inner) {
    // a tile whose halo lies inside the grid (or inside the padded band): no wrap or mirror, two
    // adjacent values per load and store (x0 - 2 and n are even; 16 bytes for FP64 storage, 8 for
    // FP32), a fixed trip count so that the loads of several pairs are in flight together
    constexpr int HP = HC / 2, NPAIR = HR * HP, IT = (NPAIR + kThreads - 1) / kThreads;
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      const int idx = threadIdx.x + k * kThreads;
      if (k + 1 < IT || idx < NPAIR) {
        const int r = idx / HP, cp = idx - r * HP;
        const int64_t gy = y0 - 2 + r, gx = x0 - 2 + 2 * cp;
        const int64_t off = (band ? gy + 2 : gy) * n + gx;
        const bool own = cbar_out && r >= 2 && r < kTY + 2 && cp >= 1 && cp < HP - 1;
        const int i0 = r * HC + 2 * cp;
        if constexpr (sizeof(T) == 4) {
          const float2 cf = *reinterpret_cast<const float2*>(cur + off);
          const float2 pf = *reinterpret_cast<const float2*>(prev + off);
          const float2 cb = make_float2(fmaf(2.0f, cf.x, -pf.x), fmaf(2.0f, cf.y, -pf.y));
          *reinterpret_cast<double2*>(sc + i0) = make_double2(widen(cf.x), widen(cf.y));
          *reinterpret_cast<double2*>(sb + i0) = make_double2(widen(cb.x), widen(cb.y));
          if (own) *reinterpret_cast<float2*>(cbar_out + gy * n + gx) = cb;
        } else {
          const double2 cd = *reinterpret_cast<const double2*>(cur + off);
          const double2 pd = *reinterpret_cast<const double2*>(prev + off);
          const double2 cb = make_double2(fma(2.0, cd.x, -pd.x), fma(2.0, cd.y, -pd.y));
          *reinterpret_cast<double2*>(sc + i0) = cd;
          *reinterpret_cast<double2*>(sb + i0) = cb;
          if (own) *reinterpret_cast<double2*>(cbar_out + gy * n + gx) = cb;
        }
      }
    }
  }
  for (int idx = inner ? HR * HC : threadIdx.x; idx < HR * HC; idx += kThreads) {
    const int r = idx / HC, c = idx - r * HC;
    const int64_t gy = y0 - 2 + r, gx = x0 - 2 + c;
    const int64_t off = band      ? (gy + 2) * n + (noflux ? mirrorn(gx, n) : wrapn(gx, n))
                        : noflux  ? static_cast<int64_t>(mirrorn(gy, n)) * n + mirrorn(gx, n)
                                  : static_cast<int64_t>(wrapn(gy, n)) * n + wrapn(gx, n);
    const double cv = widen(cur[off]);
    sc[idx] = cv;
    // cbar_out (the step's C^{n+1} buffer, non-null for the full-grid step): the tile's own Cbar,
    // which the fused update then reads instead of forming it again from C^n and C^{n-1}
    const bool own = cbar_out && r >= 2 && r < kTY + 2 && c >= 2 && c < kTX + 2;
    if constexpr (sizeof(T) == 4) {
      const float cb = fmaf(2.0f, cur[off], -prev[off]);  // as the FP32 update forms Cbar
      sb[idx] = widen(cb);
      if (own) cbar_out[gy * n + gx] = cb;
    } else {
      const double cb = fma(2.0, cv, -prev[off]);  // one FP64 instruction (2 cv - p as two adds is two)
      sb[idx] = cb;
      if (own) cbar_out[gy * n + gx] = cb;
    }
  }
  __syncthreads();
  __shared__ __align__(16) unsigned s_red[kThreads / 32];
  auto lap5 = [&](const double* t, int i, int pitch) {
    return (t[i - pitch] + t[i + pitch]) + (t[i - 1] + t[i + 1]) - 4.0 * t[i];
  };
  // digit sums of the 5-point Laplacian at i of a split tile (int2 digits over t's slots)
  auto lap5_digits = [&](const double* t, int i, int pitch, int& q0, int& q1) {
    const int2* d = reinterpret_cast<const int2*>(t);
    const int2 u = d[i - pitch], v = d[i + pitch], w = d[i - 1], x = d[i + 1], c = d[i];
    q0 = (u.x + v.x) + (w.x + x.x) - 4 * c.x;
    q1 = (u.y + v.y) + (w.y + x.y) - 4 * c.y;
  };
  if (rhs) {
    // Both 5-point Laplacians as exact integer-digit sums (weights 1, 1, 1, 1, -4; 28-bit digits, which
    // hold every bit of a value within a factor 8 of its tile's largest, so neighbouring tiles,
    // which evaluate Z on each other's border, agree on it to 2^-56 of the tile's scale and the sum
    // of the Laplacian over the grid stays zero to that level: mass is conserved), each scaled with
    // one FP64 FMA; the first one's scaling carries -a, and the cubic term N joins its digit sum
    // as an integer (cubic_q2), so the FP64 pipe keeps only Cbar, Z, the second scaling,
    // C^n - C^{n-1} and the final combination (5.3 FP64 operations per point).  A tile whose values
    // leave the digit range takes the FP64 formula for that Laplacian; a warp with a point outside
    // cubic_ok's ranges forms N in FP64.
    // the one-FMA scaling of a digit sum by m 2^(G - 56) (ixi_consts); false: the FP64 formula
    double* cb = sb;
    double* zt = sb;  // Z takes Cbar's place (held in registers until every thread has read Cbar)
    const double* cn = sc;
    {
      const int te = static_cast<int>(ixd::ix_tile_max_hi<kThreads, HR * HC>(cb, s_red) >> 20);
      uint32_t w[4];
      const bool dig = ixd::ixi_consts<28>(am51, -1.5 * am51, te, w);  // uniform over the block
      float ih = 0.0f, il = 0.0f;
      const bool cub = dig && te != 0 && cubic_scaled(cinv, te, ih, il);  // uniform too
      if (dig) {
        ixd::ixi_split_tile<kThreads, HR * HC, 28>(cb, te);
        __syncthreads();
      }
      constexpr int NZ = (ZR * ZC + kThreads - 1) / kThreads;
      double zv[NZ];
      // Z point k of this thread: the Laplacian's digit sums and u (a point past the tile reads
      // the first one; its result is not stored)
      auto zpoint = [&](int k, int& q0, int& q1, double& u) {
        int idx = threadIdx.x + k * kThreads;
        if (idx >= ZR * ZC) idx = 0;
        const int r = idx / ZC, c = idx - r * ZC;
        const int hidx = (r + 1) * HC + (c + 1);
        lap5_digits(cb, hidx, HC, q0, q1);
        u = cn[hidx];
      };
      if (cub) {
#pragma unroll
        for (int k = 0; k < NZ; k += 2) {  // two points per packed cubic term
          const int k1 = k + 1 < NZ ? k + 1 : k;
          int a0, a1, b0, b1;
          double u0, u1;
          zpoint(k, a0, a1, u0);
          zpoint(k1, b0, b1, u1);
          float h0, l0, h1, l1;
          split_hl(u0, h0, l0);
          split_hl(u1, h1, l1);
          int2 qa, qb;
          float2 qh;
          cubic_q2(make_float2(h0, h1), make_float2(l0, l1), ih, il, qa, qb, qh);
          const bool ok = cubic_ok(u0, te, qh.x, a0) && cubic_ok(u1, te, qh.y, b0);
          double z0, z1;
          if (__all_sync(0xffffffffu, ok)) {
            z0 = ixd::ixi_combine<28>(a0, a1, w, qa.x, qb.x);
            z1 = ixd::ixi_combine<28>(b0, b1, w, qa.y, qb.y);
          } else {
            z0 = fma(alpha, fma(u0 * u0, u0, -u0), ixd::ixi_combine<28>(a0, a1, w));
            z1 = fma(alpha, fma(u1 * u1, u1, -u1), ixd::ixi_combine<28>(b0, b1, w));
          }
          zv[k] = z0;
          if (k + 1 < NZ) zv[k + 1] = z1;
        }
      } else {
#pragma unroll
        for (int k = 0; k < NZ; ++k) {
          const int idx = threadIdx.x + k * kThreads;
          if (k + 1 < NZ || idx < ZR * ZC) {
            const int r = idx / ZC, c = idx - r * ZC;
            const int hidx = (r + 1) * HC + (c + 1);
            double lap_a;  // -a * Laplacian(Cbar)
            if (dig) {
              int q0, q1;
              lap5_digits(cb, hidx, HC, q0, q1);
              lap_a = ixd::ixi_combine<28>(q0, q1, w);
            } else {
              lap_a = -a * lap5(cb, hidx, HC);
            }
            const double u = cn[hidx];
            zv[k] = fma(alpha, fma(u * u, u, -u), lap_a);
          }
        }
      }
      __syncthreads();  // every thread is done with Cbar
#pragma unroll
      for (int k = 0; k < NZ; ++k) {
        const int idx = threadIdx.x + k * kThreads;
        if (k + 1 < NZ || idx < ZR * ZC) zt[idx] = zv[k];
      }
      __syncthreads();
    }
    {
      const int te = static_cast<int>(ixd::ix_tile_max_hi<kThreads, ZR * ZC>(zt, s_red) >> 20);
      uint32_t w[4];
      const bool dig = ixd::ixi_consts<28>(1.0, -1.5, te, w);
      if (dig) {
        ixd::ixi_split_tile<kThreads, ZR * ZC, 28>(zt, te);
        __syncthreads();
      }
      for (int idx = threadIdx.x; idx < kTY * kTX; idx += kThreads) {
        const int r = idx / kTX, c = idx - r * kTX;
        const int zidx = (r + 1) * ZC + (c + 1);
        const int hidx = (r + 2) * HC + (c + 2);
        double lap_z;
        if (dig) {
          int q0, q1;
          lap5_digits(zt, zidx, ZC, q0, q1);
          lap_z = ixd::ixi_combine<28>(q0, q1, w);
        } else {
          lap_z = lap5(zt, zidx, ZC);
        }
        const int64_t o = (y0 + r) * n + x0 + c;
        const double diff = cn[hidx] - widen(prev[band ? o + 2 * n : o]);  // C^n - C^{n-1}
        rhs[o] = fma(-2.0 / 3.0, diff, lap_z);
      }
    }
  }
  if (partials) {
    // Mass sum C and free-energy density sum (1/4)(C^2 - 1)^2 + (gamma / 2h^2)(|D+x C|^2 + |D+y C|^2)
    // (Eq. 1 with forward differences).  The gradient part is summed by parts: over the periodic
    // grid, and with the even reflection of the no-flux boundary, the sum of the squared forward
    // differences equals -sum C Lap5(C) (Lap5 the unscaled 5-point Laplacian, reading the staged
    // halo).  Lap5(C) is an exact digit sum scaled by one FP64 FMA, so a point costs 5 FP64
    // operations instead of 9; only the grid total (the sum over all blocks, or over all bands
    // with their halos) equals the forward-difference sum, not each block's share.
    __syncthreads();  // sb (Cbar, then Z) is no longer read: it takes C's digits
    const int te = static_cast<int>(ixd::ix_tile_max_hi<kThreads, HR * HC>(sc, s_red) >> 20);
    uint32_t w4[4];
    const bool dig = ixd::ixi_consts<28>(1.0, -1.5, te, w4);  // uniform over the block
    if (dig) {
      constexpr int NP = HR * HC / 2;
      const double2* q = reinterpret_cast<const double2*>(sc);
      int4* qi = reinterpret_cast<int4*>(sb);
      for (int k = threadIdx.x; k < NP; k += kThreads) {
        const double2 v = q[k];
        const int2 a0 = ixd::ixi_split<28>(v.x, te), a1 = ixd::ixi_split<28>(v.y, te);
        qi[k] = make_int4(a0.x, a0.y, a1.x, a1.y);
      }
      __syncthreads();
    }
    double* out2 = partials + 2 * (static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x);
    const int G = te - 1022;  // the tile's values lie below 2^G
    if (dig && G >= -3 && G <= 3) {
      // Each thread's share in exact integer arithmetic on the digit grid: u = U 2^(G-56) with
      // U = d0 2^28 + d1 (every bit of a value within a factor 8 of the tile's largest), and
      // Lap5(u) = L 2^(G-56) with L = q0 2^28 + q1 the exact digit sums.  Per point, only 32 x 32
      // -> 64-bit multiply-adds into 64-bit sums:
      //   mass      sum d0, sum d1;
      //   U L       sum d0 q0, sum (d0 q1 + d1 q0), sum d1 q1;
      //   u^2 - 1   W = round((U^2 - 2^(112-2G)) / 2^61) (units 2^(2G-51), |W| <= 2^57 + 1), from
      //             A = d0^2 - 2^(56-2G) and B = 2 d0 d1 + floor(d1^2 / 2^28) as
      //             (A >> 5) + ((A mod 32) 2^28 + B + 2^32) >> 33 (d1^2's dropped bits are below
      //             2^-33 of W's unit);
      //   W^2       with W = Wh 2^29 + Wl: sum Wh^2, sum Wh Wl, sum Wl^2.
      // Every sum of the thread's 8 points stays below 2^63; each is joined once in 128 bits, the
      // block reduces them in integers, and thread 0 converts the block's totals to FP64.  No FP64
      // operation per point or per thread (the formula below takes 5 per point, and its FP64
      // shuffle reduction 10 per thread).
      int s0 = 0, s1 = 0;
      long long g2 = 0, g1 = 0, g0 = 0, w2 = 0, w1 = 0, w0 = 0;
      const long long K56 = 1ll << (56 - 2 * G);
      const int2* dg = reinterpret_cast<const int2*>(sb);
      for (int idx = threadIdx.x; idx < kTY * kTX; idx += kThreads) {
        const int r = idx / kTX, c = idx - r * kTX;
        const int hidx = (r + 2) * HC + (c + 2);
        const int2 d = dg[hidx];
        int q0, q1;
        lap5_digits(sb, hidx, HC, q0, q1);
        s0 += d.x;
        s1 += d.y;
        g2 += static_cast<long long>(d.x) * q0;
        g1 += static_cast<long long>(d.x) * q1 + static_cast<long long>(d.y) * q0;
        g0 += static_cast<long long>(d.y) * q1;
        const long long A = static_cast<long long>(d.x) * d.x - K56;
        const long long B = static_cast<long long>(d.x) * (2 * d.y) +
                            static_cast<long long>(static_cast<unsigned long long>(static_cast<unsigned>(d.y)) * static_cast<unsigned>(d.y) >> 28);
        const long long W = (A >> 5) + ((((A & 31) << 28) + B + (1ll << 32)) >> 33);
        const int wh = static_cast<int>(W >> 29), wl = static_cast<int>(W & ((1ll << 29) - 1));
        w2 += static_cast<long long>(wh) * wh;
        w1 += static_cast<long long>(wh) * wl;
        w0 += static_cast<long long>(wl) * wl;
      }
      const __int128 sg = (static_cast<__int128>(g2) << 56) + (static_cast<__int128>(g1) << 28) + g0;
      const __int128 sw = (static_cast<__int128>(w2) << 58) + (static_cast<__int128>(w1) << 30) + w0;
      block_reduce_int(s0, s1, sg, sw, G, half_gamma_over_h2, out2);
    } else {
      double m = 0.0, ew = 0.0, eg = 0.0;
      for (int idx = threadIdx.x; idx < kTY * kTX; idx += kThreads) {
        const int r = idx / kTX, c = idx - r * kTX;
        const int hidx = (r + 2) * HC + (c + 2);
        const double u = sc[hidx];
        double lap;
        if (dig) {
          int q0, q1;
          lap5_digits(sb, hidx, HC, q0, q1);
          lap = ixd::ixi_combine<28>(q0, q1, w4);
        } else {
          lap = lap5(sc, hidx, HC);
        }
        const double w = fma(u, u, -1.0);
        m += u;
        ew = fma(w, w, ew);
        eg = fma(u, lap, eg);
      }
      block_reduce2<T>(m, fma(0.25, ew, -half_gamma_over_h2 * eg), out2);
    }
  }
}

// Fixed-order sum of the per-block partials -> out2 = (h^2 sum C, h^2 sum energy density).
__global__ void k_reduce_final(const double* __restrict__ partials, int nblocks, double h2,
                               double* __restrict__ out2) {
  __shared__ double sm[256], se[256];
  double m = 0.0, e = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 256) {
    m += partials[2 * b];
    e += partials[2 * b + 1];
  }
  sm[threadIdx.x] = m;
  se[threadIdx.x] = e;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[threadIdx.x] += sm[threadIdx.x + s];
      se[threadIdx.x] += se[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = h2 * sm[0];
    out2[1] = h2 * se[0];
  }
}

// 32-byte global accesses (one whole sector per thread and instruction)
__device__ __forceinline__ void ld_v4(const double* p, double& a, double& b, double& c, double& d) {
  asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a), "=d"(b), "=d"(c), "=d"(d) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_v4(double* p, double a, double b, double c, double d) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(a), "d"(b), "d"(c), "d"(d) : "memory");
}

// A batch of kU line elements starting at `at` (element stride es): when the line is contiguous
// (rows; `at` is then a multiple of kU) 32-byte accesses where both buffers of the kernel are
// 32-byte aligned (wide), else 16-byte ones; strided scalars for the other direction.  A thread of
// the row solves walks its own row, so a warp's access touches 32 rows: the 32-byte form fetches a
// whole sector per thread and instruction.
template <typename IT, bool CONTIG>
__device__ __forceinline__ void load_batch(const IT* __restrict__ p, int64_t at, int64_t es, double (&v)[8],
                                           bool wide = false) {
  if constexpr (CONTIG && sizeof(IT) == 8) {
    if (wide) {
      ld_v4(p + at, v[0], v[1], v[2], v[3]);
      ld_v4(p + at + 4, v[4], v[5], v[6], v[7]);
      return;
    }
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      const double2 d = *reinterpret_cast<const double2*>(p + at + u);
      v[u] = d.x;
      v[u + 1] = d.y;
    }
  } else if constexpr (CONTIG) {
#pragma unroll
    for (int u = 0; u < 8; u += 4) {
      const float4 f = *reinterpret_cast<const float4*>(p + at + u);
      v[u] = widen(f.x); v[u + 1] = widen(f.y); v[u + 2] = widen(f.z); v[u + 3] = widen(f.w);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = widen(p[at + u * es]);
  }
}
template <bool CONTIG>
__device__ __forceinline__ void store_batch(double* __restrict__ p, int64_t at, int64_t es, const double (&v)[8],
                                            bool wide = false) {
  if constexpr (CONTIG) {
    if (wide) {
      st_v4(p + at, v[0], v[1], v[2], v[3]);
      st_v4(p + at + 4, v[4], v[5], v[6], v[7]);
      return;
    }
#pragma unroll
    for (int u = 0; u < 8; u += 2) *reinterpret_cast<double2*>(p + at + u) = make_double2(v[u], v[u + 1]);
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) p[at + u * es] = v[u];
  }
}

// Phase 1: A g = b on chunk p of a line (LU forward then backward), g over the scratch.
// Coefficients (negated / pre-scaled): nl1, nl2, dinv, nu1, nu2 at coef[0..5m).  Elements are
// processed in register batches of kU so that a batch's loads are in flight together.
// NF: no-flux tables, one set of 9 m coefficients per chunk type.
template <typename IT, bool CONTIG, bool NF>
__global__ void __launch_bounds__(kSolveThreads)
    k_solve_local(const IT* __restrict__ in, double* __restrict__ G, double* __restrict__ bnd,
                  const double* __restrict__ coef, int64_t n, int P, int m, int64_t line_stride,
                  int64_t elem_stride, int p0 = 0, int Pl = -1) {
  // chunks p0 .. p0 + Pl - 1 of every line (all P of them by default); the data, G and bnd hold
  // only those, indexed from the first
  if (Pl < 0) Pl = P;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * Pl) return;
  const int64_t line = t % n;
  const int pl = static_cast<int>(t / n);
  const int p = p0 + pl;
  const int64_t es = CONTIG ? 1 : elem_stride;
  if constexpr (NF) coef += static_cast<int64_t>(chunk_type(p, P)) * 9 * m;
  const double* nl1 = coef;
  const double* nl2 = coef + m;
  const double* dinv = coef + 2 * m;
  const double* nu1 = coef + 3 * m;
  const double* nu2 = coef + 4 * m;
  const int64_t base = line * line_stride + static_cast<int64_t>(pl) * m * es;
  // rows: base is a multiple of kU elements (m and the line stride are multiples of 64)
  const bool wide = CONTIG && sizeof(IT) == 8 &&
                    ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(G)) & 31u) == 0;
  double y1 = 0.0, y2 = 0.0;
  for (int k0 = 0; k0 < m; k0 += kU) {
    double v[kU];
    load_batch<IT, CONTIG>(in, base + k0 * es, es, v, wide);
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const double y = fma(__ldg(nl1 + k0 + u), y1, fma(__ldg(nl2 + k0 + u), y2, v[u]));
      v[u] = y;
      y2 = y1;
      y1 = y;
    }
    store_batch<CONTIG>(G, base + k0 * es, es, v, wide);
  }
  double g1 = 0.0, g2 = 0.0, g_last = 0.0, g_last2 = 0.0;
  for (int k0 = m - kU; k0 >= 0; k0 -= kU) {
    double v[kU];
    load_batch<double, CONTIG>(G, base + k0 * es, es, v, wide);
#pragma unroll
    for (int u = kU - 1; u >= 0; --u) {
      const int k = k0 + u;
      const double g = fma(__ldg(nu1 + k), g1, fma(__ldg(nu2 + k), g2, v[u] * __ldg(dinv + k)));
      v[u] = g;
      g2 = g1;
      g1 = g;
    }
    if (k0 == m - kU) {
      g_last2 = v[kU - 2];
      g_last = v[kU - 1];
    }
    store_batch<CONTIG>(G, base + k0 * es, es, v, wide);
  }
  // chunk-end values: k = 0, 1 are g1, g2 after the loop; k = m-2, m-1 kept from the first batch
  double* b = bnd + static_cast<int64_t>(pl) * 4 * n + line;
  b[0] = g1;
  b[n] = g2;
  b[2 * n] = g_last2;
  b[3 * n] = g_last;
}

// Phase 2: end values of the neighbouring chunks from the block-circulant inverse (staged in
// shared memory), then the spike correction.  MODE 0 writes w (FP64); MODE 1 writes
// C^{n+1} = 2 C^n - C^{n-1} + x (for FP32 storage 2 C^n - C^{n-1} is formed in FP32: its one
// rounding, <= 2^-24 |Cbar|, is of the size of the rounding of the stored result).
// NF: no-flux tables (per chunk type) and the dense 4P x 4P chunk-end inverse, read through the
// read-only cache; the line's first chunk has no left neighbour, its last no right one.
template <int MODE, typename T, bool CONTIG, bool NF>
__global__ void __launch_bounds__(kSolveThreads)
    k_solve_correct(const double* __restrict__ G, const double* __restrict__ bnd,
                    const double* __restrict__ coef, const double* __restrict__ K, int64_t n, int P,
                    int m, int64_t line_stride, int64_t elem_stride, double* __restrict__ w_out,
                    const T* __restrict__ cur, const T* __restrict__ prev, T* __restrict__ next, int p0 = 0,
                    int Pl = -1) {
  // chunks p0 .. p0 + Pl - 1 of every line (all P by default): G, w_out and the fields hold only
  // those, indexed from the first; bnd holds the end values of all P chunks
  extern __shared__ double sK[];
  if (Pl < 0) Pl = P;
  if constexpr (!NF) {
    for (int i = threadIdx.x; i < 16 * P; i += blockDim.x) sK[i] = K[i];
    __syncthreads();
  }
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * Pl) return;
  const int64_t line = t % n;
  const int pl = static_cast<int>(t / n);
  const int p = p0 + pl;
  const int64_t es = CONTIG ? 1 : elem_stride;
  double t0 = 0.0, t1 = 0.0, h0 = 0.0, h1 = 0.0;
  if constexpr (NF) {
    coef += static_cast<int64_t>(chunk_type(p, P)) * 9 * m;
    const int64_t N4 = 4 * static_cast<int64_t>(P);
    const bool left = p > 0, right = p + 1 < P;
    const double* Kt = left ? K + (4 * static_cast<int64_t>(p - 1) + 2) * N4 : K;  // rows of x_{p-1}[m-2], [m-1]
    const double* Kh = right ? K + (4 * static_cast<int64_t>(p + 1)) * N4 : K;     // rows of x_{p+1}[0], [1]
    for (int q = 0; q < P; ++q) {
      const double* b = bnd + static_cast<int64_t>(q) * 4 * n + line;
      const double g0 = b[0], g1 = b[n], g2 = b[2 * n], g3 = b[3 * n];
      if (left) {
        const double* r2 = Kt + 4 * q;
        const double* r3 = r2 + N4;
        t0 = fma(__ldg(r2), g0, fma(__ldg(r2 + 1), g1, fma(__ldg(r2 + 2), g2, fma(__ldg(r2 + 3), g3, t0))));
        t1 = fma(__ldg(r3), g0, fma(__ldg(r3 + 1), g1, fma(__ldg(r3 + 2), g2, fma(__ldg(r3 + 3), g3, t1))));
      }
      if (right) {
        const double* r0 = Kh + 4 * q;
        const double* r1 = r0 + N4;
        h0 = fma(__ldg(r0), g0, fma(__ldg(r0 + 1), g1, fma(__ldg(r0 + 2), g2, fma(__ldg(r0 + 3), g3, h0))));
        h1 = fma(__ldg(r1), g0, fma(__ldg(r1 + 1), g1, fma(__ldg(r1 + 2), g2, fma(__ldg(r1 + 3), g3, h1))));
      }
    }
  } else {
    const int pm = (p + P - 1) % P, pp = (p + 1) % P;
    for (int q = 0; q < P; ++q) {
      const double* b = bnd + static_cast<int64_t>(q) * 4 * n + line;
      const double g0 = b[0], g1 = b[n], g2 = b[2 * n], g3 = b[3 * n];
      const double* Kt = sK + ((pm - q + P) % P) * 16;  // K_{(p-1)-q}: rows 2, 3 give t_{p-1}
      const double* Kh = sK + ((pp - q + P) % P) * 16;  // K_{(p+1)-q}: rows 0, 1 give h_{p+1}
      t0 = fma(Kt[8], g0, fma(Kt[9], g1, fma(Kt[10], g2, fma(Kt[11], g3, t0))));
      t1 = fma(Kt[12], g0, fma(Kt[13], g1, fma(Kt[14], g2, fma(Kt[15], g3, t1))));
      h0 = fma(Kh[0], g0, fma(Kh[1], g1, fma(Kh[2], g2, fma(Kh[3], g3, h0))));
      h1 = fma(Kh[4], g0, fma(Kh[5], g1, fma(Kh[6], g2, fma(Kh[7], g3, h1))));
    }
  }
  const double* sl0 = coef + 5 * m;
  const double* sl1 = coef + 6 * m;
  const double* sr0 = coef + 7 * m;
  const double* sr1 = coef + 8 * m;
  const int64_t base = line * line_stride + static_cast<int64_t>(pl) * m * es;
  const bool wide = CONTIG && MODE == 0 &&
                    ((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(w_out)) & 31u) == 0;
  for (int k0 = 0; k0 < m; k0 += kU) {
    double x[kU];
    load_batch<double, CONTIG>(G, base + k0 * es, es, x, wide);
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int k = k0 + u;
      x[u] = fma(-__ldg(sl0 + k), t0, fma(-__ldg(sl1 + k), t1,
             fma(-__ldg(sr0 + k), h0, fma(-__ldg(sr1 + k), h1, x[u]))));
    }
    if constexpr (MODE == 0) {
      store_batch<CONTIG>(w_out, base + k0 * es, es, x, wide);
    } else {
      // next holds Cbar = 2 C^n - C^{n-1}, written there by this step's right-hand side kernel
      // (FP32 storage: formed in FP32, one rounding of the size of the result's own); C^{n+1} =
      // Cbar + v replaces it element by element
      if constexpr (sizeof(T) == 4) {
        // one FP64 add of x, then the round-to-nearest-even narrowing on the integer pipe (this
        // kernel is FP64-bound, and a conversion instruction would take an FP64 issue slot)
        float cb[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) cb[u] = next[base + (k0 + u) * es];
#pragma unroll
        for (int u = 0; u < kU; ++u) next[base + (k0 + u) * es] = narrow_rn(widen(cb[u]) + x[u]);
      } else {
        double cb[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) cb[u] = next[base + (k0 + u) * es];
#pragma unroll
        for (int u = 0; u < kU; ++u) store_as<T>(next + base + (k0 + u) * es, cb[u] + x[u]);
      }
    }
  }
}

// ---- host-side precomputation ---------------------------------------------------------------

// LU of the m x m pentadiagonal Toeplitz block, rows (a, -4a, 1+6a, -4a, a), no pivoting
// (the block is symmetric positive definite).  L unit lower with bands l1, l2; U with d, u1, u2.
void block_lu(int m, double a, std::vector<double>& l1, std::vector<double>& l2,
              std::vector<double>& d, std::vector<double>& u1, std::vector<double>& u2) {
  l1.assign(m, 0.0); l2.assign(m, 0.0); d.assign(m, 0.0); u1.assign(m, 0.0); u2.assign(m, 0.0);
  for (int k = 0; k < m; ++k) {
    const double sub2 = k >= 2 ? a : 0.0;
    const double sub1 = k >= 1 ? -4.0 * a : 0.0;
    l2[k] = k >= 2 ? sub2 / d[k - 2] : 0.0;
    l1[k] = k >= 1 ? (sub1 - (k >= 2 ? l2[k] * u1[k - 2] : 0.0)) / d[k - 1] : 0.0;
    d[k] = 1.0 + 6.0 * a - (k >= 2 ? l2[k] * u2[k - 2] : 0.0) - (k >= 1 ? l1[k] * u1[k - 1] : 0.0);
    u1[k] = k + 1 < m ? -4.0 * a - (k >= 1 ? l1[k] * u2[k - 1] : 0.0) : 0.0;
    u2[k] = k + 2 < m ? a : 0.0;
  }
}

// LU (no pivoting) of an m x m pentadiagonal block given by its bands: sub2[k] = A(k, k-2),
// sub1[k] = A(k, k-1), diag[k], sup1[k] = A(k, k+1), sup2[k] = A(k, k+2).
void penta_lu(int m, const std::vector<double>& sub2, const std::vector<double>& sub1,
              const std::vector<double>& diag, const std::vector<double>& sup1,
              const std::vector<double>& sup2, std::vector<double>& l1, std::vector<double>& l2,
              std::vector<double>& d, std::vector<double>& u1, std::vector<double>& u2) {
  l1.assign(m, 0.0); l2.assign(m, 0.0); d.assign(m, 0.0); u1.assign(m, 0.0); u2.assign(m, 0.0);
  for (int k = 0; k < m; ++k) {
    l2[k] = k >= 2 ? sub2[k] / d[k - 2] : 0.0;
    l1[k] = k >= 1 ? (sub1[k] - (k >= 2 ? l2[k] * u1[k - 2] : 0.0)) / d[k - 1] : 0.0;
    d[k] = diag[k] - (k >= 2 ? l2[k] * u2[k - 2] : 0.0) - (k >= 1 ? l1[k] * u1[k - 1] : 0.0);
    u1[k] = k + 1 < m ? sup1[k] - (k >= 1 ? l1[k] * u2[k - 1] : 0.0) : 0.0;
    u2[k] = k + 2 < m ? sup2[k] : 0.0;
  }
}

void block_solve(int m, const std::vector<double>& l1, const std::vector<double>& l2,
                 const std::vector<double>& d, const std::vector<double>& u1,
                 const std::vector<double>& u2, std::vector<double>& x) {
  for (int k = 0; k < m; ++k) {
    if (k >= 1) x[k] -= l1[k] * x[k - 1];
    if (k >= 2) x[k] -= l2[k] * x[k - 2];
  }
  for (int k = m - 1; k >= 0; --k) {
    if (k + 1 < m) x[k] -= u1[k] * x[k + 1];
    if (k + 2 < m) x[k] -= u2[k] * x[k + 2];
    x[k] /= d[k];
  }
}

// Gauss-Jordan inverse with partial pivoting (dense, small), then two steps of Newton refinement
// K <- K + K (I - R K) whose residual I - R K is accumulated with error-free products and sums
// (FMA and TwoSum), so it is exact to rounding although it is far smaller than R K: the
// chunk-end system's condition number grows with a, and the plain inverse's rounding (~cond * eps)
// went straight into every corrected value (the solver's backward error was 3.9e-13 of
// (1 + 16 a) |x| at n = 4096 with no-flux boundaries; refined it is 2.6e-15).
bool invert(int N, std::vector<double>& Min, std::vector<double>& inv) {
  const std::vector<double> R = Min;
  std::vector<double>& M = Min;
  inv.assign(static_cast<size_t>(N) * N, 0.0);
  for (int i = 0; i < N; ++i) inv[static_cast<size_t>(i) * N + i] = 1.0;
  for (int c = 0; c < N; ++c) {
    int piv = c;
    for (int r = c + 1; r < N; ++r)
      if (std::fabs(M[static_cast<size_t>(r) * N + c]) > std::fabs(M[static_cast<size_t>(piv) * N + c])) piv = r;
    if (M[static_cast<size_t>(piv) * N + c] == 0.0) return false;
    if (piv != c)
      for (int k = 0; k < N; ++k) {
        std::swap(M[static_cast<size_t>(c) * N + k], M[static_cast<size_t>(piv) * N + k]);
        std::swap(inv[static_cast<size_t>(c) * N + k], inv[static_cast<size_t>(piv) * N + k]);
      }
    const double s = 1.0 / M[static_cast<size_t>(c) * N + c];
    for (int k = 0; k < N; ++k) {
      M[static_cast<size_t>(c) * N + k] *= s;
      inv[static_cast<size_t>(c) * N + k] *= s;
    }
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const double f = M[static_cast<size_t>(r) * N + c];
      if (f == 0.0) continue;
      for (int k = 0; k < N; ++k) {
        M[static_cast<size_t>(r) * N + k] -= f * M[static_cast<size_t>(c) * N + k];
        inv[static_cast<size_t>(r) * N + k] -= f * inv[static_cast<size_t>(c) * N + k];
      }
    }
  }
  std::vector<double> E(static_cast<size_t>(N) * N), C(static_cast<size_t>(N) * N);
  for (int it = 0; it < 2; ++it) {
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < N; ++c) {  // E = I - R K, each entry as an unevaluated sum hi + lo
        double hi = r == c ? 1.0 : 0.0, lo = 0.0;
        for (int k = 0; k < N; ++k) {
          const double p = -R[static_cast<size_t>(r) * N + k] * inv[static_cast<size_t>(k) * N + c];
          const double pe = std::fma(-R[static_cast<size_t>(r) * N + k], inv[static_cast<size_t>(k) * N + c], -p);
          const double t = hi + p, bb = t - hi;
          lo += (hi - (t - bb)) + (p - bb) + pe;
          hi = t;
        }
        E[static_cast<size_t>(r) * N + c] = hi + lo;
      }
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < N; ++c) {  // C = K E
        double acc = 0.0;
        for (int k = 0; k < N; ++k) acc = std::fma(inv[static_cast<size_t>(r) * N + k], E[static_cast<size_t>(k) * N + c], acc);
        C[static_cast<size_t>(r) * N + c] = acc;
      }
    for (size_t q = 0; q < C.size(); ++q) inv[q] += C[q];
  }
  return true;
}

int build_tables_periodic(int64_t n, int P, double a, std::vector<double>& coef, std::vector<double>& K) {
  const int m = static_cast<int>(n / P);
  std::vector<double> l1, l2, d, u1, u2;
  block_lu(m, a, l1, l2, d, u1, u2);
  coef.assign(static_cast<size_t>(9) * m, 0.0);
  for (int k = 0; k < m; ++k) {
    coef[k] = -l1[k];
    coef[m + k] = -l2[k];
    coef[2 * m + k] = 1.0 / d[k];
    coef[3 * m + k] = -u1[k] / d[k];
    coef[4 * m + k] = -u2[k] / d[k];
  }
  // spikes: responses to the two values before (t) and after (h) the chunk
  std::vector<double> s[4];
  for (int c = 0; c < 4; ++c) s[c].assign(m, 0.0);
  s[0][0] = a;                          // S_L column for x_{p-1}[m-2]
  s[1][0] = -4.0 * a; s[1][1] = a;      // S_L column for x_{p-1}[m-1]
  s[2][m - 2] = a; s[2][m - 1] = -4.0 * a;  // S_R column for x_{p+1}[0]
  s[3][m - 1] = a;                      // S_R column for x_{p+1}[1]
  for (int c = 0; c < 4; ++c) block_solve(m, l1, l2, d, u1, u2, s[c]);
  for (int c = 0; c < 4; ++c)
    for (int k = 0; k < m; ++k) coef[static_cast<size_t>(5 + c) * m + k] = s[c][k];
  // block-circulant system for u_p = (x_p[0], x_p[1], x_p[m-2], x_p[m-1])
  const int rows[4] = {0, 1, m - 2, m - 1};
  const int N4 = 4 * P;
  std::vector<double> R(static_cast<size_t>(N4) * N4, 0.0), Ri;
  for (int i = 0; i < N4; ++i) R[static_cast<size_t>(i) * N4 + i] = 1.0;
  for (int p = 0; p < P; ++p) {
    const int pm = (p + P - 1) % P, pp = (p + 1) % P;
    for (int r = 0; r < 4; ++r) {
      const size_t row = static_cast<size_t>(4 * p + r) * N4;
      R[row + 4 * pm + 2] += s[0][rows[r]];
      R[row + 4 * pm + 3] += s[1][rows[r]];
      R[row + 4 * pp + 0] += s[2][rows[r]];
      R[row + 4 * pp + 1] += s[3][rows[r]];
    }
  }
  if (!invert(N4, R, Ri)) return set_error(CS_EINVAL, "Cahn-Hilliard chunk system is singular");
  K.assign(static_cast<size_t>(16) * P, 0.0);
  for (int dd = 0; dd < P; ++dd)  // K_d = block (d, 0) of the inverse
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) K[static_cast<size_t>(dd) * 16 + r * 4 + c] = Ri[static_cast<size_t>(4 * dd + r) * N4 + c];
  return CS_OK;
}

// No-flux tables: for each chunk type t (bit 0: the line's first chunk, bit 1: its last) the LU
// of the chunk block of L = I + a D4 (reflected rows at the line's ends) and the four spikes, at
// coef[9 m t ..]; K = the dense inverse of the 4P x 4P chunk-end system, row-major.
int build_tables_noflux(int64_t n, int P, double a, std::vector<double>& coef, std::vector<double>& K) {
  const int m = static_cast<int>(n / P);
  coef.assign(static_cast<size_t>(4) * 9 * m, 0.0);
  std::vector<double> spk[4][4];  // [type][spike]
  for (int t = 0; t < 4; ++t) {
    std::vector<double> sub2(m, a), sub1(m, -4.0 * a), diag(m, 1.0 + 6.0 * a), sup1(m, -4.0 * a), sup2(m, a);
    if (t & 1) {  // rows 0, 1 of the line: (1 + 2a, -3a, a), (-3a, 1 + 6a, -4a, a)
      diag[0] = 1.0 + 2.0 * a;
      sup1[0] = -3.0 * a;
      sub1[1] = -3.0 * a;
    }
    if (t & 2) {  // rows n-2, n-1: mirrored
      diag[m - 1] = 1.0 + 2.0 * a;
      sub1[m - 1] = -3.0 * a;
      sup1[m - 2] = -3.0 * a;
    }
    std::vector<double> l1, l2, d, u1, u2;
    penta_lu(m, sub2, sub1, diag, sup1, sup2, l1, l2, d, u1, u2);
    double* c = coef.data() + static_cast<size_t>(9) * m * t;
    for (int k = 0; k < m; ++k) {
      c[k] = -l1[k];
      c[m + k] = -l2[k];
      c[2 * m + k] = 1.0 / d[k];
      c[3 * m + k] = -u1[k] / d[k];
      c[4 * m + k] = -u2[k] / d[k];
    }
    for (int q = 0; q < 4; ++q) spk[t][q].assign(m, 0.0);
    if (!(t & 1)) {  // couplings to the previous chunk's last two values
      spk[t][0][0] = a;
      spk[t][1][0] = -4.0 * a; spk[t][1][1] = a;
    }
    if (!(t & 2)) {  // couplings to the next chunk's first two values
      spk[t][2][m - 2] = a; spk[t][2][m - 1] = -4.0 * a;
      spk[t][3][m - 1] = a;
    }
    for (int q = 0; q < 4; ++q) {
      block_solve(m, l1, l2, d, u1, u2, spk[t][q]);
      for (int k = 0; k < m; ++k) c[static_cast<size_t>(5 + q) * m + k] = spk[t][q][k];
    }
  }
  const int rows[4] = {0, 1, m - 2, m - 1};
  const int N4 = 4 * P;
  std::vector<double> R(static_cast<size_t>(N4) * N4, 0.0);
  for (int i = 0; i < N4; ++i) R[static_cast<size_t>(i) * N4 + i] = 1.0;
  for (int p = 0; p < P; ++p) {
    const int t = (p == 0 ? 1 : 0) | (p == P - 1 ? 2 : 0);
    for (int r = 0; r < 4; ++r) {
      const size_t row = static_cast<size_t>(4 * p + r) * N4;
      if (p > 0) {
        R[row + 4 * (p - 1) + 2] += spk[t][0][rows[r]];
        R[row + 4 * (p - 1) + 3] += spk[t][1][rows[r]];
      }
      if (p + 1 < P) {
        R[row + 4 * (p + 1) + 0] += spk[t][2][rows[r]];
        R[row + 4 * (p + 1) + 1] += spk[t][3][rows[r]];
      }
    }
  }
  if (!invert(N4, R, K)) return set_error(CS_EINVAL, "Cahn-Hilliard chunk system is singular");
  return CS_OK;
}

int build_tables(int64_t n, int P, double a, bool noflux, std::vector<double>& coef, std::vector<double>& K) {
  return noflux ? build_tables_noflux(n, P, a, coef, K) : build_tables_periodic(n, P, a, coef, K);
}

// Valid partition: P divides n, chunks of at least 16 points in whole register batches.
bool valid_chunks(int64_t n, int P) {
  return P >= 1 && P <= 64 && n % P == 0 && (n / P) >= 16 && (n / P) % kU == 0;
}

int default_chunks(int64_t n) {
  // enough independent (line, chunk) threads to fill the GPU, while the chunk-end system
  // (16 P^2 / n FP64 operations per point) stays at most 4 per point
  int P = 1;
  while (n * P < 65536 && valid_chunks(n, 2 * P) && 16.0 * (2 * P) * (2 * P) / n <= 4.0) P *= 2;
  return P;
}

// FP64 tiles (C^n, Cbar: halo 2; Z: halo 1), for either storage type.
size_t rhs_smem_bytes() {
  return 8 * (2 * (kTY + 4) * (kTX + 4));  // C^n and Cbar (Z reuses Cbar's space)
}

template <typename T> int set_rhs_attr() {
  static bool done = false;
  if (!done) {
    const int bytes = static_cast<int>(rhs_smem_bytes());
    CS_CUDA_TRY(cudaFuncSetAttribute(k_ch_rhs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done = true;
  }
  return CS_OK;
}

template <typename T>
int launch_rhs(CHPlan* p, bool with_rhs, double* partials, cudaStream_t s) {
  int rc = set_rhs_attr<T>();
  if (rc != CS_OK) return rc;
  dim3 grid(static_cast<unsigned>(p->n / kTX), static_cast<unsigned>(p->n / kTY));
  const T* cur = static_cast<const T*>(p->field[p->icur]);
  const T* prev = static_cast<const T*>(p->field[p->iprev]);
  double* rhs = with_rhs ? p->A : nullptr;
  T* cbar = with_rhs ? static_cast<T*>(p->field[p->inext]) : nullptr;
  k_ch_rhs<T><<<grid, kThreads, rhs_smem_bytes(), s>>>(cur, prev, rhs, p->n, p->alpha, p->a,
                                                        0.5 * p->gamma / (p->h * p->h), partials, p->noflux,
                                                        ixd::ixi_round51(-p->a),
                                                        cubic_inv(p->alpha, ixd::ixi_round51(-p->a)), 0, cbar);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

template <typename T, bool NF>
void launch_solves(CHPlan* p, cudaStream_t s) {
  const int64_t n = p->n;
  const unsigned sgrid = static_cast<unsigned>((n * p->P + kSolveThreads - 1) / kSolveThreads);
  const size_t ksmem = NF ? 0 : static_cast<size_t>(16) * p->P * sizeof(double);
  // x-sweep: lines are rows (line stride n, element stride 1)
  k_solve_local<double, true, NF><<<sgrid, kSolveThreads, 0, s>>>(p->A, p->B, p->bnd, p->coef, n, p->P,
                                                                  p->m, n, 1);
  k_solve_correct<0, T, true, NF><<<sgrid, kSolveThreads, ksmem, s>>>(p->B, p->bnd, p->coef, p->K, n, p->P,
                                                                      p->m, n, 1, p->A, nullptr, nullptr, nullptr);
  // y-sweep: lines are columns (line stride 1, element stride n), update fused
  k_solve_local<double, false, NF><<<sgrid, kSolveThreads, 0, s>>>(p->A, p->B, p->bnd, p->coef, n, p->P,
                                                                   p->m, 1, n);
  k_solve_correct<1, T, false, NF><<<sgrid, kSolveThreads, ksmem, s>>>(
      p->B, p->bnd, p->coef, p->K, n, p->P, p->m, 1, n, nullptr,
      static_cast<const T*>(p->field[p->icur]), static_cast<const T*>(p->field[p->iprev]),
      static_cast<T*>(p->field[p->inext]));
}

template <typename T>
int launch_step(CHPlan* p, double* partials, cudaStream_t s) {
  int rc = launch_rhs<T>(p, true, partials, s);
  if (rc != CS_OK) return rc;
  if (p->noflux) launch_solves<T, true>(p, s);
  else launch_solves<T, false>(p, s);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(4);
  return CS_OK;
}

void rotate(CHPlan* p) {
  const int old_prev = p->iprev;
  p->iprev = p->icur;
  p->icur = p->inext;
  p->inext = old_prev;
  ++p->steps;
}

int reduce_current(CHPlan* p, double* out2, cudaStream_t s) {
  int rc = p->storage == CS_F32 ? launch_rhs<float>(p, false, p->partials, s)
                                : launch_rhs<double>(p, false, p->partials, s);
  if (rc != CS_OK) return rc;
  k_reduce_final<<<1, 256, 0, s>>>(p->partials, p->rhs_blocks, p->h * p->h, out2);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

void free_plan(CHPlan* p) {
  if (!p) return;
  drop_graphs(p);
  cudaFree(p->A); cudaFree(p->B); cudaFree(p->bnd); cudaFree(p->coef); cudaFree(p->K);
  cudaFree(p->partials); cudaFree(p->inv); cudaFree(p->diag);
  delete p;
}

}  // namespace

int ch_create(CHPlan** out, const cs_ch_desc* d, void* prev, void* cur, void* next) {
  *out = nullptr;
  if (!d) return set_error(CS_EINVAL, "null Cahn-Hilliard description");
  if (d->n < 64 || d->n % 64 != 0 || d->n > 65536)
    return set_error(CS_EINVAL, "n must be a multiple of 64 in [64, 65536]");
  if (d->storage != CS_F64 && d->storage != CS_F32) return set_error(CS_EINVAL, "storage must be CS_F64 or CS_F32");
  if (d->boundary != CS_CH_PERIODIC && d->boundary != CS_CH_NOFLUX)
    return set_error(CS_EINVAL, "boundary must be CS_CH_PERIODIC or CS_CH_NOFLUX");
  if (!(d->D > 0) || !(d->gamma >= 0) || !(d->dt > 0) || !std::isfinite(d->D) || !std::isfinite(d->gamma) || !std::isfinite(d->dt))
    return set_error(CS_EINVAL, "D > 0, gamma >= 0, dt > 0 and finite are required");
  if (!prev || !cur || !next) return set_error(CS_EINVAL, "null field buffer");
  const size_t eb = d->storage == CS_F32 ? 4 : 8;
  const size_t bytes = static_cast<size_t>(d->n) * d->n * eb;
  void* f[3] = {prev, cur, next};
  for (int i = 0; i < 3; ++i) {
    if (reinterpret_cast<uintptr_t>(f[i]) % eb) return set_error(CS_EINVAL, "fields must be aligned to the element size");
    for (int j = i + 1; j < 3; ++j) {
      const char* a = static_cast<const char*>(f[i]);
      const char* b = static_cast<const char*>(f[j]);
      if (a < b + bytes && b < a + bytes) return set_error(CS_EALIAS, "the three fields must not overlap");
    }
  }
  CHPlan* p = new (std::nothrow) CHPlan;
  if (!p) return set_error(CS_ENOMEM, "out of host memory");
  memset(p, 0, sizeof *p);
  p->n = d->n;
  p->storage = d->storage;
  p->noflux = d->boundary == CS_CH_NOFLUX;
  p->D = d->D; p->gamma = d->gamma; p->dt = d->dt;
  p->h = 2.0 * M_PI / static_cast<double>(d->n);
  const double h2 = p->h * p->h;
  p->a = (2.0 / 3.0) * d->D * d->gamma * d->dt / (h2 * h2);
  p->alpha = (2.0 / 3.0) * d->D * d->dt / h2;
  int P = default_chunks(d->n);
  int choice;
  char key[96];
  snprintf(key, sizeof key, "ch|%s%s|n%lld|sm%d", d->storage == CS_F32 ? "f32" : "f64",
           p->noflux ? "|noflux" : "", (long long)d->n, num_sms());
  if (tune_lookup(key, &choice) && valid_chunks(d->n, choice)) P = choice;
  p->P = P;
  p->m = static_cast<int>(d->n / P);
  p->field[0] = prev; p->field[1] = cur; p->field[2] = next;
  p->iprev = 0; p->icur = 1; p->inext = 2;
  p->rhs_blocks = static_cast<int>((d->n / kTX) * (d->n / kTY));
  std::vector<double> coef, K;
  int rc = build_tables(d->n, P, p->a, p->noflux != 0, coef, K);
  if (rc != CS_OK) { free_plan(p); return rc; }
  const size_t nn = static_cast<size_t>(d->n) * d->n;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&p->A, nn * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->B, nn * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->bnd, static_cast<size_t>(4) * P * d->n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->coef, coef.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->K, K.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->partials, static_cast<size_t>(2) * p->rhs_blocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(p->coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->K, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_plan(p);
    return e == cudaErrorMemoryAllocation ? set_error(CS_ENOMEM, "Cahn-Hilliard workspace: %s", cudaGetErrorString(e))
                                          : cuda_error(e, "Cahn-Hilliard workspace");
  }
  rc = d->storage == CS_F32 ? set_rhs_attr<float>() : set_rhs_attr<double>();  // before any capture
  if (rc != CS_OK) { free_plan(p); return rc; }
  *out = p;
  return CS_OK;
}

void drop_graphs(CHPlan* p) {
  for (int i = 0; i < 3; ++i) {
    if (p->graph3[i]) cudaGraphExecDestroy(p->graph3[i]);
    p->graph3[i] = nullptr;
  }
}

// Captures three consecutive steps starting at the current rotation phase into a graph (the
// buffers return to the same roles after three steps, so the graph replays as is).
int capture_three(CHPlan* p, cudaGraphExec_t* out) {
  cudaStream_t cap;
  CS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  const int ip = p->iprev, ic = p->icur, in = p->inext;
  const int64_t steps = p->steps;
  const int64_t before = cs_launch_count();
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? CS_OK : cuda_error(e, "cudaStreamBeginCapture");
  for (int k = 0; k < 3 && rc == CS_OK; ++k) {
    rc = p->storage == CS_F32 ? launch_step<float>(p, nullptr, cap) : launch_step<double>(p, nullptr, cap);
    rotate(p);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  cudaStreamDestroy(cap);
  p->iprev = ip; p->icur = ic; p->inext = in; p->steps = steps;  // capture ran nothing
  p->graph_kernels = static_cast<int>(cs_launch_count() - before);
  count_launches(-p->graph_kernels);
  if (rc != CS_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (e2 != cudaSuccess) return cuda_error(e2, "cudaStreamEndCapture");
  cudaError_t e3 = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) { *out = nullptr; return cuda_error(e3, "cudaGraphInstantiate"); }
  return CS_OK;
}

int ch_step(CHPlan* p, int64_t nsteps, double* h_mass, double* h_energy, cudaStream_t s) {
  if (nsteps < 0) return set_error(CS_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return CS_OK;
  const bool want = h_mass || h_energy;
  if (!want) {  // blocks of three steps replay a captured graph (fewer launch gaps)
    while (nsteps >= 3) {
      cudaGraphExec_t& g = p->graph3[p->icur];
      if (!g) {
        int rc = capture_three(p, &g);
        if (rc != CS_OK) return rc;
      }
      CS_CUDA_TRY(cudaGraphLaunch(g, s));
      count_launches(p->graph_kernels);
      rotate(p); rotate(p); rotate(p);
      nsteps -= 3;
    }
    for (; nsteps > 0; --nsteps) {
      int rc = p->storage == CS_F32 ? launch_step<float>(p, nullptr, s) : launch_step<double>(p, nullptr, s);
      if (rc != CS_OK) return rc;
      rotate(p);
    }
    return CS_OK;
  }
  if (p->inv_cap < nsteps) {
    if (p->inv) cudaFree(p->inv);
    p->inv = nullptr;
    p->inv_cap = 0;
    cudaError_t e = cudaMalloc(&p->inv, static_cast<size_t>(2) * nsteps * sizeof(double));
    if (e != cudaSuccess) return cuda_error(e, "invariant buffer");
    p->inv_cap = nsteps;
  }
  for (int64_t st = 0; st < nsteps; ++st) {
    // the RHS kernel of step st reads C^n = the field after step st-1: reduce it on the way
    double* part = st > 0 ? p->partials : nullptr;
    int rc = p->storage == CS_F32 ? launch_step<float>(p, part, s) : launch_step<double>(p, part, s);
    if (rc != CS_OK) return rc;
    if (part) {
      // partials were consumed into a fixed-order sum before the next RHS overwrites them
      k_reduce_final<<<1, 256, 0, s>>>(p->partials, p->rhs_blocks, p->h * p->h, p->inv + 2 * (st - 1));
      CS_CUDA_TRY(cudaGetLastError());
      count_launches(1);
    }
    rotate(p);
  }
  int rc = reduce_current(p, p->inv + 2 * (nsteps - 1), s);
  if (rc != CS_OK) return rc;
  std::vector<double> h(static_cast<size_t>(2) * nsteps);
  CS_CUDA_TRY(cudaMemcpyAsync(h.data(), p->inv, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CS_CUDA_TRY(cudaStreamSynchronize(s));
  for (int64_t st = 0; st < nsteps; ++st) {
    if (h_mass) h_mass[st] = h[2 * st];
    if (h_energy) h_energy[st] = h[2 * st + 1];
  }
  return CS_OK;
}

int ch_invariants(CHPlan* p, double* mass, double* energy, cudaStream_t s) {
  if (p->inv_cap < 1) {
    cudaError_t e = cudaMalloc(&p->inv, 2 * sizeof(double));
    if (e != cudaSuccess) return cuda_error(e, "invariant buffer");
    p->inv_cap = 1;
  }
  int rc = reduce_current(p, p->inv, s);
  if (rc != CS_OK) return rc;
  double h[2];
  CS_CUDA_TRY(cudaMemcpyAsync(h, p->inv, sizeof h, cudaMemcpyDeviceToHost, s));
  CS_CUDA_TRY(cudaStreamSynchronize(s));
  if (mass) *mass = h[0];
  if (energy) *energy = h[1];
  return CS_OK;
}

namespace {

// ---- coarsening measures (Sec. 5.1, "Numerical Results") ---------------------------------------
//   s(t)   = 1 / (1 - <C^2>), <.> the spatial average by Simpson's rule on the periodic grid
//            (weights 2, 4, 2, 4, ... per direction: the end point 2 pi is the start point);
//   k_1(t) = sum_k |C^(k)|^2 / sum_k |k|^-1 |C^(k)|^2 over the discrete wavenumbers, k = 0 left out
//            (the k-space integrals with their common measure cancelled).
// The 2D DFT is two passes of a radix-2 FFT (one CTA per row, the row in shared memory): the
// first transforms the rows of C and writes them transposed into the (A, B) = (re, im) scratch,
// the second transforms those rows (the columns of C) and sums the spectrum.  All FP64.

constexpr int kDiagThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kDiagThreads)
    k_simpson_rows(const T* __restrict__ c, int64_t n, double* __restrict__ partials) {
  const int64_t j = blockIdx.x;  // one row per block
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kDiagThreads) {
    const double v = widen(c[j * n + i]);
    acc += ((i & 1) ? 4.0 : 2.0) * v * v;
  }
  __shared__ double red[kDiagThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kDiagThreads / 32; ++w) r += red[w];
    partials[j] = ((j & 1) ? 4.0 : 2.0) * r;
  }
}

// In-place radix-2 decimation-in-time FFT of the n = 2^logn points in (xr, xi) (shared memory,
// loaded in bit-reversed order); tw holds exp(-2 pi i t / n) for t < n / 2.
__device__ __forceinline__ void fft_smem(double* xr, double* xi, int n, int logn, const double2* __restrict__ tw) {
  for (int len = 2, stride = n >> 1; len <= n; len <<= 1, stride >>= 1) {
    const int half = len >> 1;
    for (int b = threadIdx.x; b < (n >> 1); b += kDiagThreads) {
      const int pos = b & (half - 1);
      const int i = (b - pos) * 2 + pos, k = i + half;
      const double2 w = tw[pos * stride];
      const double vr = w.x * xr[k] - w.y * xi[k];
      const double vi = w.x * xi[k] + w.y * xr[k];
      const double ur = xr[i], ui = xi[i];
      xr[i] = ur + vr;
      xi[i] = ui + vi;
      xr[k] = ur - vr;
      xi[k] = ui - vi;
    }
    __syncthreads();
  }
  (void)logn;
}

__device__ __forceinline__ int bit_reverse(int t, int logn) { return static_cast<int>(__brev(static_cast<unsigned>(t)) >> (32 - logn)); }

// Pass 1: the FFT of row j of C, written as column j of (re, im).
template <typename T>
__global__ void __launch_bounds__(kDiagThreads)
    k_fft_rows(const T* __restrict__ c, int n, int logn, const double2* __restrict__ tw,
               double* __restrict__ re, double* __restrict__ im) {
  extern __shared__ double xs[];
  double* xr = xs;
  double* xi = xs + n;
  const int64_t j = blockIdx.x;
  for (int t = threadIdx.x; t < n; t += kDiagThreads) {
    const int r = bit_reverse(t, logn);
    xr[r] = widen(c[j * n + t]);
    xi[r] = 0.0;
  }
  __syncthreads();
  fft_smem(xr, xi, n, logn, tw);
  for (int k = threadIdx.x; k < n; k += kDiagThreads) {
    re[static_cast<int64_t>(k) * n + j] = xr[k];
    im[static_cast<int64_t>(k) * n + j] = xi[k];
  }
}

// Pass 2: the FFT of row kx of (re, im) (column kx of the row transforms) gives C^(kx, ky) for
// every ky; the block sums |C^|^2 and |k|^-1 |C^|^2 (k = 0 left out) into partials[2 kx + 0/1].
__global__ void __launch_bounds__(kDiagThreads)
    k_fft_cols_spectrum(const double* __restrict__ re, const double* __restrict__ im, int n, int logn,
                        const double2* __restrict__ tw, double* __restrict__ partials) {
  extern __shared__ double xs[];
  double* xr = xs;
  double* xi = xs + n;
  const int kx = blockIdx.x;
  for (int t = threadIdx.x; t < n; t += kDiagThreads) {
    const int r = bit_reverse(t, logn);
    xr[r] = re[static_cast<int64_t>(kx) * n + t];
    xi[r] = im[static_cast<int64_t>(kx) * n + t];
  }
  __syncthreads();
  fft_smem(xr, xi, n, logn, tw);
  const double fx = kx <= n / 2 ? kx : kx - n;
  double num = 0.0, den = 0.0;
  for (int ky = threadIdx.x; ky < n; ky += kDiagThreads) {
    if (kx == 0 && ky == 0) continue;
    const double fy = ky <= n / 2 ? ky : ky - n;
    const double pw = xr[ky] * xr[ky] + xi[ky] * xi[ky];
    num += pw;
    den += pw / sqrt(fx * fx + fy * fy);
  }
  __shared__ double red[2][kDiagThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, off);
    den += __shfl_down_sync(0xffffffffu, den, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kDiagThreads / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partials[2 * kx] = a;
    partials[2 * kx + 1] = b;
  }
}

// Fixed-order sums of the partials: out[0] = sum of n Simpson row sums, out[1], out[2] = the two
// spectral sums.
__global__ void k_coarsening_final(const double* __restrict__ simpson, const double* __restrict__ spec,
                                   int n, double* __restrict__ out) {
  __shared__ double r[3][256];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    a += simpson[i];
    b += spec[2 * i];
    c += spec[2 * i + 1];
  }
  r[0][threadIdx.x] = a;
  r[1][threadIdx.x] = b;
  r[2][threadIdx.x] = c;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int q = 0; q < 3; ++q) r[q][threadIdx.x] += r[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) out[q] = r[q][0];
}

}  // namespace

int ch_coarsening(CHPlan* p, double* s_out, double* k1_out, cudaStream_t st) {
  if (p->noflux) return set_error(CS_EUNSUPPORTED, "the coarsening measures are defined on the periodic grid");
  const int64_t n = p->n;
  int logn = 0;
  while ((int64_t(1) << logn) < n) ++logn;
  if ((int64_t(1) << logn) != n) return set_error(CS_EUNSUPPORTED, "coarsening measures need n a power of two");
  const size_t smem = 2 * static_cast<size_t>(n) * sizeof(double);
  if (smem > 200 * 1024) return set_error(CS_EUNSUPPORTED, "n = %lld too large for the shared-memory FFT", (long long)n);
  // diag: [0, n) twiddles as n/2 (re, im) pairs, [n, 2n) Simpson row sums, [2n, 4n) spectrum sums, 4 results
  if (!p->diag) {
    std::vector<double> tw(static_cast<size_t>(n));
    for (int64_t t = 0; t < n / 2; ++t) {
      const double ang = -2.0 * M_PI * static_cast<double>(t) / static_cast<double>(n);
      tw[2 * t] = std::cos(ang);
      tw[2 * t + 1] = std::sin(ang);
    }
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, (4 * static_cast<size_t>(n) + 4) * sizeof(double));
    if (e != cudaSuccess)
      return e == cudaErrorMemoryAllocation ? set_error(CS_ENOMEM, "coarsening buffers: %s", cudaGetErrorString(e))
                                            : cuda_error(e, "coarsening buffers");
    e = cudaMemcpyAsync(d, tw.data(), n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_error(e, "coarsening twiddles");
    }
    p->diag = d;
  }
  // the attribute is per function and process-wide: set it for this plan's n on every call
  CS_CUDA_TRY(cudaFuncSetAttribute(k_fft_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  CS_CUDA_TRY(cudaFuncSetAttribute(k_fft_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  CS_CUDA_TRY(cudaFuncSetAttribute(k_fft_cols_spectrum, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  const double2* tw = reinterpret_cast<const double2*>(p->diag);
  double* simpson = p->diag + n;
  double* spec = p->diag + 2 * n;
  double* res = p->diag + 4 * n;
  const unsigned grid = static_cast<unsigned>(n);
  if (p->storage == CS_F32) {
    const float* c = static_cast<const float*>(p->field[p->icur]);
    k_simpson_rows<float><<<grid, kDiagThreads, 0, st>>>(c, n, simpson);
    k_fft_rows<float><<<grid, kDiagThreads, smem, st>>>(c, static_cast<int>(n), logn, tw, p->A, p->B);
  } else {
    const double* c = static_cast<const double*>(p->field[p->icur]);
    k_simpson_rows<double><<<grid, kDiagThreads, 0, st>>>(c, n, simpson);
    k_fft_rows<double><<<grid, kDiagThreads, smem, st>>>(c, static_cast<int>(n), logn, tw, p->A, p->B);
  }
  k_fft_cols_spectrum<<<grid, kDiagThreads, smem, st>>>(p->A, p->B, static_cast<int>(n), logn, tw, spec);
  k_coarsening_final<<<1, 256, 0, st>>>(simpson, spec, static_cast<int>(n), res);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(4);
  double h[3];
  CS_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, st));
  CS_CUDA_TRY(cudaStreamSynchronize(st));
  const double mean_c2 = h[0] / (9.0 * static_cast<double>(n) * static_cast<double>(n));
  if (s_out) *s_out = 1.0 / (1.0 - mean_c2);
  if (k1_out) *k1_out = h[1] / h[2];
  return CS_OK;
}

int ch_fields(CHPlan* p, void** prev, void** cur, int64_t* steps) {
  if (prev) *prev = p->field[p->iprev];
  if (cur) *cur = p->field[p->icur];
  if (steps) *steps = p->steps;
  return CS_OK;
}

namespace {

// (Re)builds the partition tables and chunk-end buffer for P chunks per line.
int set_partition(CHPlan* p, int P) {
  std::vector<double> coef, K;
  int rc = build_tables(p->n, P, p->a, p->noflux != 0, coef, K);
  if (rc != CS_OK) return rc;
  double *bnd = nullptr, *dcoef = nullptr, *dK = nullptr;
  cudaError_t e = cudaMalloc(&bnd, static_cast<size_t>(4) * P * p->n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dcoef, coef.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dK, K.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(dcoef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dK, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(bnd); cudaFree(dcoef); cudaFree(dK);
    return cuda_error(e, "Cahn-Hilliard partition tables");
  }
  drop_graphs(p);
  cudaFree(p->bnd); cudaFree(p->coef); cudaFree(p->K);
  p->bnd = bnd; p->coef = dcoef; p->K = dK;
  p->P = P;
  p->m = static_cast<int>(p->n / P);
  return CS_OK;
}

}  // namespace

// Times one step for every valid chunk count (1 .. 64 chunks per line) from the plan's current
// state, keeps the fastest, records it in the tuning table, and restores the fields.
int ch_autotune(CHPlan* p, cudaStream_t s) {
  const size_t eb = p->storage == CS_F32 ? 4 : 8;
  const size_t bytes = static_cast<size_t>(p->n) * p->n * eb;
  void* save[2] = {nullptr, nullptr};
  CS_CUDA_TRY(cudaMalloc(&save[0], bytes));
  cudaError_t e = cudaMalloc(&save[1], bytes);
  if (e != cudaSuccess) { cudaFree(save[0]); return cuda_error(e, "autotune state copy"); }
  const int ip = p->iprev, ic = p->icur, in = p->inext;
  const int64_t steps = p->steps;
  e = cudaMemcpyAsync(save[0], p->field[ip], bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(save[1], p->field[ic], bytes, cudaMemcpyDeviceToDevice, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int rc = e == cudaSuccess ? CS_OK : cuda_error(e, "autotune setup");
  int best = p->P;
  float best_ms = 1e30f;
  for (int P = 1; P <= 64 && rc == CS_OK; P *= 2) {
    if (!valid_chunks(p->n, P)) continue;
    rc = set_partition(p, P);
    if (rc != CS_OK) break;
    rc = ch_step(p, 1, nullptr, nullptr, s);  // warm-up
    if (rc != CS_OK) break;
    cudaEventRecord(e0, s);
    rc = ch_step(p, 2, nullptr, nullptr, s);
    cudaEventRecord(e1, s);
    if (rc != CS_OK) break;
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { rc = cuda_error(e, "autotune timing"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = P; }
  }
  if (rc == CS_OK) rc = set_partition(p, best);
  // restore the state the caller had
  p->iprev = ip; p->icur = ic; p->inext = in; p->steps = steps;
  cudaMemcpyAsync(p->field[ip], save[0], bytes, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(p->field[ic], save[1], bytes, cudaMemcpyDeviceToDevice, s);
  cudaStreamSynchronize(s);
  cudaFree(save[0]); cudaFree(save[1]);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != CS_OK) return rc;
  char key[96];
  snprintf(key, sizeof key, "ch|%s%s|n%lld|sm%d", p->storage == CS_F32 ? "f32" : "f64",
           p->noflux ? "|noflux" : "", (long long)p->n, num_sms());
  tune_store(key, best);
  return CS_OK;
}

int ch_set_fields(CHPlan* p, void* prev, void* cur, void* next) {
  if (!prev || !cur || !next) return set_error(CS_EINVAL, "null field buffer");
  const size_t eb = p->storage == CS_F32 ? 4 : 8;
  const size_t bytes = static_cast<size_t>(p->n) * p->n * eb;
  void* f[3] = {prev, cur, next};
  for (int i = 0; i < 3; ++i) {
    if (reinterpret_cast<uintptr_t>(f[i]) % eb) return set_error(CS_EINVAL, "fields must be aligned to the element size");
    for (int j = i + 1; j < 3; ++j) {
      const char* a = static_cast<const char*>(f[i]);
      const char* b = static_cast<const char*>(f[j]);
      if (a < b + bytes && b < a + bytes) return set_error(CS_EALIAS, "the three fields must not overlap");
    }
  }
  drop_graphs(p);
  p->field[0] = prev; p->field[1] = cur; p->field[2] = next;
  p->iprev = 0; p->icur = 1; p->inext = 2;
  p->steps = 0;
  return CS_OK;
}

int ch_config(CHPlan* p, int32_t* chunks, int32_t* chunk_len) {
  if (chunks) *chunks = p->P;
  if (chunk_len) *chunk_len = p->m;
  return CS_OK;
}

void ch_destroy(CHPlan* p) { free_plan(p); }

// ---- a row band of a grid decomposed over several GPUs ----------------------------------------------
// The pieces of the ADI step that a caller runs on its own band of rows (Sec. 6.2's decomposition),
// periodic or with no-flux boundaries:
// the right-hand side and invariant sums of the band from padded C^n, C^{n-1} (2 halo rows each
// side, exchanged by the caller), line solves along the rows of a buffer (the x lines of the band,
// or after a transpose the y lines of a band of columns), and the update C^{n+1} = Cbar + v on the
// band.  The kernels are the full-grid step's own, so the decomposed step gives the same values.
struct CHBand {
  int64_t n, rows;
  int storage;
  int noflux;  // CS_CH_NOFLUX: mirrored columns, non-cyclic line solves
  double D, gamma, dt, h, a, alpha;
  int P, m;
  double* coef;
  double* K;
  double* B;         // rows * n scratch (local solutions)
  double* bnd;       // 4 * P * rows chunk-end values
  double* partials;  // 2 per RHS block
  int rhs_blocks;
};

namespace {
template <typename T>
__global__ void __launch_bounds__(256)
    k_ch_band_update(const T* __restrict__ prev, const T* __restrict__ cur, const double* __restrict__ v,
                     T* __restrict__ next, int64_t n, int64_t count) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t o = i + 2 * n;  // padded row r + 2
  if constexpr (sizeof(T) == 4) {
    const float cb = fmaf(2.0f, cur[o], -prev[o]);  // as the full-grid update forms it
    next[o] = narrow_rn(widen(cb) + v[i]);
  } else {
    next[o] = fma(2.0, cur[o], -prev[o]) + v[i];
  }
}

void free_band(CHBand* b) {
  if (!b) return;
  cudaFree(b->coef); cudaFree(b->K); cudaFree(b->B); cudaFree(b->bnd); cudaFree(b->partials);
  delete b;
}
}  // namespace

// The partition (chunks per line) cs_ch_create picks for a description: the autotuner's choice
// for it when one is recorded, else the default.
static int band_partition(const cs_ch_desc* d) {
  int P = default_chunks(d->n), choice;
  char key[96];
  snprintf(key, sizeof key, "ch|%s%s|n%lld|sm%d", d->storage == CS_F32 ? "f32" : "f64",
           d->boundary == CS_CH_NOFLUX ? "|noflux" : "", (long long)d->n, num_sms());
  if (tune_lookup(key, &choice) && valid_chunks(d->n, choice)) P = choice;
  return P;
}

int ch_band_create(CHBand** out, const cs_ch_desc* d, int64_t rows) {
  *out = nullptr;
  if (!d) return set_error(CS_EINVAL, "null Cahn-Hilliard description");
  if (d->boundary != CS_CH_PERIODIC && d->boundary != CS_CH_NOFLUX)
    return set_error(CS_EINVAL, "boundary must be CS_CH_PERIODIC or CS_CH_NOFLUX");
  if (d->n < 64 || d->n % 64 != 0 || d->n > 65536) return set_error(CS_EINVAL, "n must be a multiple of 64 in [64, 65536]");
  if (rows < kTY || rows % kTY != 0 || rows > d->n) return set_error(CS_EINVAL, "band rows must be a multiple of %d in [%d, n]", kTY, kTY);
  if (d->storage != CS_F64 && d->storage != CS_F32) return set_error(CS_EINVAL, "storage must be CS_F64 or CS_F32");
  if (!(d->D > 0) || !(d->gamma >= 0) || !(d->dt > 0) || !std::isfinite(d->D) || !std::isfinite(d->gamma) || !std::isfinite(d->dt))
    return set_error(CS_EINVAL, "D > 0, gamma >= 0, dt > 0 and finite are required");
  CHBand* b = new (std::nothrow) CHBand;
  if (!b) return set_error(CS_ENOMEM, "out of host memory");
  memset(b, 0, sizeof *b);
  b->n = d->n; b->rows = rows; b->storage = d->storage;
  b->noflux = d->boundary == CS_CH_NOFLUX;
  b->D = d->D; b->gamma = d->gamma; b->dt = d->dt;
  b->h = 2.0 * M_PI / static_cast<double>(d->n);
  const double h2 = b->h * b->h;
  b->a = (2.0 / 3.0) * d->D * d->gamma * d->dt / (h2 * h2);
  b->alpha = (2.0 / 3.0) * d->D * d->dt / h2;
  const int P = band_partition(d);  // the full-grid plan's partition
  b->P = P;
  b->m = static_cast<int>(d->n / P);
  b->rhs_blocks = static_cast<int>((d->n / kTX) * (rows / kTY));
  std::vector<double> coef, K;
  int rc = build_tables(d->n, P, b->a, b->noflux != 0, coef, K);
  if (rc != CS_OK) { free_band(b); return rc; }
  cudaError_t e = cudaMalloc(&b->coef, coef.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->K, K.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->B, static_cast<size_t>(rows) * d->n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->bnd, static_cast<size_t>(4) * P * rows * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->partials, static_cast<size_t>(2) * b->rhs_blocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(b->coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->K, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_band(b);
    return e == cudaErrorMemoryAllocation ? set_error(CS_ENOMEM, "band workspace: %s", cudaGetErrorString(e))
                                          : cuda_error(e, "band workspace");
  }
  rc = d->storage == CS_F32 ? set_rhs_attr<float>() : set_rhs_attr<double>();
  if (rc != CS_OK) { free_band(b); return rc; }
  *out = b;
  return CS_OK;
}

int ch_band_rhs(CHBand* b, const void* prev, const void* cur, double* rhs, double* sums, cudaStream_t s) {
  if (!prev || !cur || (!rhs && !sums)) return set_error(CS_EINVAL, "null buffer");
  dim3 grid(static_cast<unsigned>(b->n / kTX), static_cast<unsigned>(b->rows / kTY));
  const double hg = 0.5 * b->gamma / (b->h * b->h);
  double* part = sums ? b->partials : nullptr;
  if (b->storage == CS_F32)
    k_ch_rhs<float><<<grid, kThreads, rhs_smem_bytes(), s>>>(static_cast<const float*>(cur), static_cast<const float*>(prev),
                                                              rhs, b->n, b->alpha, b->a, hg, part, b->noflux,
                                                              ixd::ixi_round51(-b->a),
                                                              cubic_inv(b->alpha, ixd::ixi_round51(-b->a)), 1, nullptr);
  else
    k_ch_rhs<double><<<grid, kThreads, rhs_smem_bytes(), s>>>(static_cast<const double*>(cur), static_cast<const double*>(prev),
                                                               rhs, b->n, b->alpha, b->a, hg, part, b->noflux,
                                                               ixd::ixi_round51(-b->a),
                                                               cubic_inv(b->alpha, ixd::ixi_round51(-b->a)), 1, nullptr);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  if (sums) {
    k_reduce_final<<<1, 256, 0, s>>>(b->partials, b->rhs_blocks, b->h * b->h, sums);
    CS_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  return CS_OK;
}

int ch_band_solve(CHBand* b, const double* in, double* out, cudaStream_t s) {
  if (!in || !out) return set_error(CS_EINVAL, "null buffer");
  const unsigned sgrid = static_cast<unsigned>((b->rows * b->P + kSolveThreads - 1) / kSolveThreads);
  // rows lines of n points, line stride n, element stride 1 (the kernels' line count is `rows`)
  if (b->noflux) {
    k_solve_local<double, true, true><<<sgrid, kSolveThreads, 0, s>>>(in, b->B, b->bnd, b->coef, b->rows, b->P,
                                                                     b->m, b->n, 1);
    k_solve_correct<0, double, true, true><<<sgrid, kSolveThreads, 0, s>>>(
        b->B, b->bnd, b->coef, b->K, b->rows, b->P, b->m, b->n, 1, out, nullptr, nullptr, nullptr);
  } else {
    const size_t ksmem = static_cast<size_t>(16) * b->P * sizeof(double);
    k_solve_local<double, true, false><<<sgrid, kSolveThreads, 0, s>>>(in, b->B, b->bnd, b->coef, b->rows, b->P,
                                                                      b->m, b->n, 1);
    k_solve_correct<0, double, true, false><<<sgrid, kSolveThreads, ksmem, s>>>(
        b->B, b->bnd, b->coef, b->K, b->rows, b->P, b->m, b->n, 1, out, nullptr, nullptr, nullptr);
  }
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(2);
  return CS_OK;
}

int ch_partition(const cs_ch_desc* d, int32_t* chunks, int32_t* chunk_len) {
  if (!d) return set_error(CS_EINVAL, "null Cahn-Hilliard description");
  if (d->n < 64 || d->n % 64 != 0 || d->n > 65536) return set_error(CS_EINVAL, "n must be a multiple of 64 in [64, 65536]");
  if (d->boundary != CS_CH_PERIODIC && d->boundary != CS_CH_NOFLUX)
    return set_error(CS_EINVAL, "boundary must be CS_CH_PERIODIC or CS_CH_NOFLUX");
  const int P = band_partition(d);
  if (chunks) *chunks = P;
  if (chunk_len) *chunk_len = static_cast<int32_t>(d->n / P);
  return CS_OK;
}

// The y lines of a band whose rows are whole chunks of those lines: chunks chunk0 .. chunk0 +
// rows / m - 1 of every column.  Phase 1 solves each of them locally (the x pass's own kernel with
// lines = the n columns, line stride 1, element stride n) into the plan's scratch and writes their
// end values to ends; phase 2, once the caller has gathered every band's end values in chunk order,
// applies the spike correction and writes v.
static int band_ycols_check(const CHBand* b, int64_t chunk0) {
  if (b->rows % b->m != 0)
    return set_error(CS_EINVAL, "band of %lld rows is not a whole number of %d-row chunks", (long long)b->rows, b->m);
  if (chunk0 < 0 || chunk0 + b->rows / b->m > b->P)
    return set_error(CS_EINVAL, "chunks %lld .. %lld outside the %d chunks of a line", (long long)chunk0,
                     (long long)(chunk0 + b->rows / b->m - 1), b->P);
  return CS_OK;
}

int ch_band_ycols_local(CHBand* b, int64_t chunk0, const double* in, double* ends, cudaStream_t s) {
  if (!in || !ends) return set_error(CS_EINVAL, "null buffer");
  int rc = band_ycols_check(b, chunk0);
  if (rc != CS_OK) return rc;
  const int Pl = static_cast<int>(b->rows / b->m);
  const unsigned sgrid = static_cast<unsigned>((b->n * Pl + kSolveThreads - 1) / kSolveThreads);
  if (b->noflux)
    k_solve_local<double, false, true><<<sgrid, kSolveThreads, 0, s>>>(in, b->B, ends, b->coef, b->n, b->P, b->m, 1,
                                                                       b->n, static_cast<int>(chunk0), Pl);
  else
    k_solve_local<double, false, false><<<sgrid, kSolveThreads, 0, s>>>(in, b->B, ends, b->coef, b->n, b->P, b->m, 1,
                                                                        b->n, static_cast<int>(chunk0), Pl);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

int ch_band_ycols_correct(CHBand* b, int64_t chunk0, const double* ends_all, double* v, cudaStream_t s) {
  if (!ends_all || !v) return set_error(CS_EINVAL, "null buffer");
  int rc = band_ycols_check(b, chunk0);
  if (rc != CS_OK) return rc;
  const int Pl = static_cast<int>(b->rows / b->m);
  const unsigned sgrid = static_cast<unsigned>((b->n * Pl + kSolveThreads - 1) / kSolveThreads);
  if (b->noflux) {
    k_solve_correct<0, double, false, true><<<sgrid, kSolveThreads, 0, s>>>(
        b->B, ends_all, b->coef, b->K, b->n, b->P, b->m, 1, b->n, v, nullptr, nullptr, nullptr,
        static_cast<int>(chunk0), Pl);
  } else {
    const size_t ksmem = static_cast<size_t>(16) * b->P * sizeof(double);
    k_solve_correct<0, double, false, false><<<sgrid, kSolveThreads, ksmem, s>>>(
        b->B, ends_all, b->coef, b->K, b->n, b->P, b->m, 1, b->n, v, nullptr, nullptr, nullptr,
        static_cast<int>(chunk0), Pl);
  }
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

int ch_band_update(CHBand* b, const void* prev, const void* cur, const double* v, void* next, cudaStream_t s) {
  if (!prev || !cur || !v || !next) return set_error(CS_EINVAL, "null buffer");
  const int64_t count = b->rows * b->n;
  const unsigned grid = static_cast<unsigned>((count + 255) / 256);
  if (b->storage == CS_F32)
    k_ch_band_update<float><<<grid, 256, 0, s>>>(static_cast<const float*>(prev), static_cast<const float*>(cur), v,
                                                 static_cast<float*>(next), b->n, count);
  else
    k_ch_band_update<double><<<grid, 256, 0, s>>>(static_cast<const double*>(prev), static_cast<const double*>(cur), v,
                                                  static_cast<double*>(next), b->n, count);
  CS_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return CS_OK;
}

void ch_band_destroy(CHBand* b) { free_band(b); }

// Host replay of the device line solver (phase 1: chunk LU forward and backward, chunk-end
// values; phase 2: neighbouring chunk ends from K, spike correction), in the kernels' order of
// operations, on the tables cs_ch_create builds, for a pseudo-random right-hand side; returns the
// backward error ||L x - b||_inf / ((1 + 16 a) ||x||_inf) of the result against the line operator
// itself (periodic: circulant (1, -4, 6, -4, 1); no-flux: reflected rows at the ends).
int ch_solver_check(int64_t n, int P, double a, bool noflux, double* residual) {
  if (!residual) return set_error(CS_EINVAL, "null residual pointer");
  if (n < 16 || n > 65536 || !valid_chunks(n, P)) return set_error(CS_EINVAL, "invalid line length / chunk count");
  if (!(a >= 0.0) || !std::isfinite(a)) return set_error(CS_EINVAL, "a must be finite and >= 0");
  std::vector<double> coef, K;
  int rc = build_tables(n, P, a, noflux, coef, K);
  if (rc != CS_OK) return rc;
  const int m = static_cast<int>(n / P);
  std::vector<double> b(n), g(n), x(n), ends(static_cast<size_t>(4) * P);
  uint64_t st = 0x9E3779B97F4A7C15ull ^ static_cast<uint64_t>(n * 131 + P);
  for (int64_t i = 0; i < n; ++i) {  // xorshift64*: values in [-1, 1)
    st ^= st >> 12; st ^= st << 25; st ^= st >> 27;
    b[i] = static_cast<double>((st * 0x2545F4914F6CDD1Dull) >> 11) * 0x1p-52 - 1.0;
  }
  auto tab = [&](int p) { return coef.data() + (noflux ? static_cast<size_t>(9) * m * chunk_type(p, P) : 0); };
  for (int p = 0; p < P; ++p) {  // phase 1
    const double* c = tab(p);
    double y1 = 0.0, y2 = 0.0;
    for (int k = 0; k < m; ++k) {
      const double y = fma(c[k], y1, fma(c[m + k], y2, b[p * m + k]));
      g[p * m + k] = y;
      y2 = y1;
      y1 = y;
    }
    double g1 = 0.0, g2 = 0.0;
    for (int k = m - 1; k >= 0; --k) {
      const double v = fma(c[3 * m + k], g1, fma(c[4 * m + k], g2, g[p * m + k] * c[2 * m + k]));
      g[p * m + k] = v;
      g2 = g1;
      g1 = v;
    }
    ends[4 * p] = g[p * m];
    ends[4 * p + 1] = g[p * m + 1];
    ends[4 * p + 2] = g[p * m + m - 2];
    ends[4 * p + 3] = g[p * m + m - 1];
  }
  const int64_t N4 = 4 * static_cast<int64_t>(P);
  for (int p = 0; p < P; ++p) {  // phase 2
    double t0 = 0.0, t1 = 0.0, h0 = 0.0, h1 = 0.0;
    for (int q = 0; q < P; ++q) {
      const double* e = ends.data() + 4 * q;
      if (noflux) {
        if (p > 0) {
          const double* r2 = K.data() + (4 * static_cast<int64_t>(p - 1) + 2) * N4 + 4 * q;
          const double* r3 = r2 + N4;
          t0 = fma(r2[0], e[0], fma(r2[1], e[1], fma(r2[2], e[2], fma(r2[3], e[3], t0))));
          t1 = fma(r3[0], e[0], fma(r3[1], e[1], fma(r3[2], e[2], fma(r3[3], e[3], t1))));
        }
        if (p + 1 < P) {
          const double* r0 = K.data() + 4 * static_cast<int64_t>(p + 1) * N4 + 4 * q;
          const double* r1 = r0 + N4;
          h0 = fma(r0[0], e[0], fma(r0[1], e[1], fma(r0[2], e[2], fma(r0[3], e[3], h0))));
          h1 = fma(r1[0], e[0], fma(r1[1], e[1], fma(r1[2], e[2], fma(r1[3], e[3], h1))));
        }
      } else {
        const double* Kt = K.data() + ((p + P - 1 - q + P) % P) * 16;
        const double* Kh = K.data() + ((p + 1 - q + P) % P) * 16;
        t0 = fma(Kt[8], e[0], fma(Kt[9], e[1], fma(Kt[10], e[2], fma(Kt[11], e[3], t0))));
        t1 = fma(Kt[12], e[0], fma(Kt[13], e[1], fma(Kt[14], e[2], fma(Kt[15], e[3], t1))));
        h0 = fma(Kh[0], e[0], fma(Kh[1], e[1], fma(Kh[2], e[2], fma(Kh[3], e[3], h0))));
        h1 = fma(Kh[4], e[0], fma(Kh[5], e[1], fma(Kh[6], e[2], fma(Kh[7], e[3], h1))));
      }
    }
    const double* c = tab(p);
    for (int k = 0; k < m; ++k)
      x[p * m + k] = fma(-c[5 * m + k], t0, fma(-c[6 * m + k], t1, fma(-c[7 * m + k], h0, fma(-c[8 * m + k], h1, g[p * m + k]))));
  }
  double rmax = 0.0, xmax = 0.0;
  auto at = [&](int64_t i) {  // periodic wrap or even reflection
    if (!noflux) return x[(i % n + n) % n];
    if (i < 0) i = -1 - i;
    if (i >= n) i = 2 * n - 1 - i;
    return x[i];
  };
  for (int64_t i = 0; i < n; ++i) {
    // L = I + a D4; D4 is the fourth difference, on the reflected line the square of the
    // reflected second difference, which reflection of x reproduces at every row
    double d2[3];
    for (int j = -1; j <= 1; ++j) d2[j + 1] = at(i + j - 1) - 2.0 * at(i + j) + at(i + j + 1);
    if (noflux) {  // D2 of the reflected line, taken again with reflection
      auto d2at = [&](int64_t k) {
        if (k < 0) k = -1 - k;
        if (k >= n) k = 2 * n - 1 - k;
        return at(k - 1) - 2.0 * at(k) + at(k + 1);
      };
      for (int j = -1; j <= 1; ++j) d2[j + 1] = d2at(i + j);
    }
    const double lx = x[i] + a * (d2[0] - 2.0 * d2[1] + d2[2]);
    rmax = std::max(rmax, std::fabs(lx - b[i]));
    xmax = std::max(xmax, std::fabs(x[i]));
  }
  *residual = rmax / ((1.0 + 16.0 * a) * std::max(xmax, 1e-300));
  return CS_OK;
}

}  // namespace cs
