// Float-pair arithmetic shared by the Jacobi kernels, the float-pair SpMV
// merge path and the mixed-stream executor (internal).  A float64 value x is carried as an unevaluated pair
// of floats (hi, lo) with x = hi + lo to ~2^-46 relative; conversions use
// integer bit operations only, because float64<->float32 conversion
// instructions issue on B300's slow float64 pipe.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ar {

constexpr double kSixth = 1.0 / 6.0;

// Unknown (i, j, k) of an N^3 grid, or 0 outside the cube (Dirichlet ghost).
__device__ __forceinline__ double at(const double* __restrict__ u, int N, int i, int j, int k) {
  if ((unsigned)i >= (unsigned)N || (unsigned)j >= (unsigned)N || (unsigned)k >= (unsigned)N) return 0.0;
  return u[((int64_t)k * N + j) * N + i];
}

// 1/6 as an unevaluated float pair.
constexpr float kSixthHi = 0.16666667163372039794921875f;           // RN(1/6)
constexpr float kSixthLo = -4.967053740534411e-09f;  // RN(1/6 - kSixthHi)

// Split x into floats (hi, lo): hi = x truncated to 24 significant bits,
// lo = the next 23 bits of the remainder (same sign as x, |lo| < ulp(hi)),
// so x = hi + lo to within 2^-46 |x|.  Integer operations plus one float add
// and one float multiply: on B300 a float64<->float32 conversion issues on
// the slow float64 pipe, and int->float conversion is avoided too (2^23 + q
// is read as a float straight from its bits).  Values outside the float-pair
// range (|x| < 2^-74, |x| >= 2^118, inf, NaN) give hi = NaN as a marker;
// +-0 gives (0, 0).
__device__ __forceinline__ float2 df_split(double x) {
  const long long b = __double_as_longlong(x);
  const unsigned h32 = (unsigned)((unsigned long long)b >> 32), l32 = (unsigned)b;
  const unsigned e = (h32 >> 20) & 0x7ffu;
  const unsigned sign = h32 & 0x80000000u;
  // exponent bits 8..0 and the top 23 significand bits; adding 2^30 rebiases
  // the 9-bit exponent field from 1023 to 127 (mod 512) for every e in range
  const unsigned hib = (__funnelshift_l(l32, h32, 3) + 0x40000000u) | sign;
  const float q = __uint_as_float(0x4b000000u | ((l32 >> 6) & 0x7fffffu)) - 8388608.0f;
  const float lo = q * __uint_as_float(((e - 942u) << 23) | sign);  // q * +-2^(e-1069)
  float2 out = make_float2(__uint_as_float(hib), lo);
  // branch-free selects: +-0 -> (0, 0); outside [2^-74, 2^118) or inf/NaN -> marker
  if (e - 949u > 191u) out = ((b << 1) == 0) ? make_float2(0.f, 0.f) : make_float2(__int_as_float(0x7fc00001), 0.f);
  return out;
}

// Exact float -> float64 by assembling the bit pattern (no conversion
// instruction).  Subnormal floats become signed zero (|f| < 2^-126 is below
// the resolution of any float-pair result here); inf/NaN become NaN.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e8 = (u >> 23) & 0xffu;
  unsigned hi = u & 0x80000000u, lo = 0u;
  if (e8 == 0xffu) {
    hi = 0x7ff80000u;
  } else if (e8 != 0u) {
    hi |= ((e8 + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    lo = u << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// v0 + ... + v5 in float-pair arithmetic as the unevaluated pair (s, c): the
// hi parts are summed exactly by a TwoSum chain, the chain's errors and the
// lo parts in plain float.
__device__ __forceinline__ void df_sum6(float2 v0, float2 v1, float2 v2, float2 v3, float2 v4, float2 v5, float& s,
                                        float& c) {
  float e;
  two_sum(v0.x, v1.x, s, c);
  two_sum(s, v2.x, s, e);
  c += e;
  two_sum(s, v3.x, s, e);
  c += e;
  two_sum(s, v4.x, s, e);
  c += e;
  two_sum(s, v5.x, s, e);
  c += e;
  c += ((v0.y + v1.y) + (v2.y + v3.y)) + (v4.y + v5.y);
}

// (v0 + ... + v5) / 6 in float-pair arithmetic: returns the unevaluated
// pair (p, pe) with p + pe = the average to ~2^-46 relative; the sum is
// multiplied by 1/6 as a float pair.
__device__ __forceinline__ float2 df_avg6(float2 v0, float2 v1, float2 v2, float2 v3, float2 v4, float2 v5) {
  float s, c;
  df_sum6(v0, v1, v2, v3, v4, v5, s, c);
  const float p = s * kSixthHi;
  float pe = fmaf(s, kSixthHi, -p);
  pe = fmaf(s, kSixthLo, pe);
  pe = fmaf(c, kSixthHi, pe);
  return make_float2(p, pe);
}

// u + alpha (v0 + ... + v5 - 6 u), the explicit heat update, in float-pair
// arithmetic as beta u + alpha sum with beta = 1 - 6 alpha: alpha = ahi + alo
// and beta = bhi + blo are float pairs, each product a pair product (the lo x
// lo term dropped), the two summed by TwoSum; absolute error ~2^-46 (|beta|
// |u| + |alpha| sum |v|), at most ~2^-46 max |v| for 0 <= alpha <= 1/6.
__device__ __forceinline__ float2 df_heat(float2 u, float2 v0, float2 v1, float2 v2, float2 v3, float2 v4, float2 v5,
                                          float ahi, float alo, float bhi, float blo) {
  float s, c;
  df_sum6(v0, v1, v2, v3, v4, v5, s, c);
  const float q = ahi * s;
  float qe = fmaf(ahi, s, -q);
  qe = fmaf(alo, s, qe);
  qe = fmaf(ahi, c, qe);
  const float r = bhi * u.x;
  float re = fmaf(bhi, u.x, -r);
  re = fmaf(blo, u.x, re);
  re = fmaf(bhi, u.y, re);
  float h, e;
  two_sum(q, r, h, e);
  e += qe + re;
  return make_float2(h, e);
}

// The two 7-point stencils: the Jacobi average (W + E + S + N + D + U) / 6
// and the explicit heat step u + alpha (W + E + S + N + D + U - 6 u).
enum Stencil { kJacobi = 0, kHeat = 1 };
struct StencilCoef {
  double alpha;    // heat: the step's alpha = kappa dt / h^2
  float ahi, alo;  // alpha as a float pair
  float bhi, blo;  // 1 - 6 alpha as a float pair
};

// float64 form; s = W + E + S + N + D + U summed in that order, u the centre
template <int ST>
__device__ __forceinline__ double stencil_f64(double u, double s, const StencilCoef& k) {
  if constexpr (ST == kJacobi)
    return s * kSixth;
  else
    return u + k.alpha * (s - 6.0 * u);
}

// float-pair form of the same update
template <int ST>
__device__ __forceinline__ float2 stencil_pair(float2 u, float2 w, float2 e, float2 so, float2 no, float2 d,
                                               float2 up, const StencilCoef& k) {
  if constexpr (ST == kJacobi)
    return df_avg6(w, e, so, no, d, up);
  else
    return df_heat(u, w, e, so, no, d, up, k.ahi, k.alo, k.bhi, k.blo);
}

__device__ __forceinline__ double pair_to_double(float2 v) { return f2d_bits(v.x) + f2d_bits(v.y); }

// f2d_bits for a finite float (no inf / NaN case): fewer operations.
__device__ __forceinline__ double f2d_finite(float f) {
  const unsigned u = __float_as_uint(f), a = u & 0x7fffffffu;
  const bool normal = a >= 0x00800000u;  // zero and subnormals become signed zero
  const unsigned hi = (u & 0x80000000u) | (normal ? (a >> 3) + 0x38000000u : 0u);
  return __hiloint2double((int)hi, normal ? (int)(u << 29) : 0);
}

// pair_to_double for a pair of finite floats.
__device__ __forceinline__ double finite_pair_to_double(float2 v) { return f2d_finite(v.x) + f2d_finite(v.y); }

// Split a product operand x into floats hi + lo (hi = x truncated to 24
// significant bits, 0 <= lo/x < 2^-23, x - hi - lo below 2^-46 |x|) with
// integer operations and one float add.  The
// range is [2^-62, 2^62) in magnitude, so that products of two operands and
// their low parts stay normal floats; +-0 gives (0, 0).  Returns false (and
// (0, 0)) for any other value: the caller redoes that work in float64.
__device__ __forceinline__ bool prod_split(double x, float& hi, float& lo) {
  const long long b = __double_as_longlong(x);
  const unsigned h32 = (unsigned)((unsigned long long)b >> 32), l32 = (unsigned)b;
  const unsigned e = (h32 >> 20) & 0x7ffu;
  const unsigned sign = h32 & 0x80000000u;
  // float exponent e - 896 lands in bits 31..23 as (e mod 512) + 128 mod 512,
  // which is e - 896 < 256 for every e in range: sign bit left clear
  const unsigned hib = (__funnelshift_l(l32, h32, 3) + 0x40000000u) | sign;
  // lo from the top 23 of the 29 remainder bits (the dropped 6 bits are below
  // 2^-46 |x|): 2^23 + q is a float read straight from its bits, so no
  // int->float conversion instruction is needed
  const float q = __uint_as_float(0x4b000000u | ((l32 >> 6) & 0x7fffffu)) - 8388608.0f;
  const float scale = __uint_as_float(((e - 942u) << 23) | sign);  // +-2^(e-1069)
  const bool ok = e - 961u < 124u;
  hi = ok ? __uint_as_float(hib) : 0.f;
  lo = ok ? q * scale : 0.f;
  return ok || ((h32 & 0x7fffffffu) | l32) == 0u;
}

// (S, C) += (p, pe) for unevaluated float pairs ("sloppy" pair addition):
// the absolute error is below ~2^-46 (|S| + |p|) whatever the signs.
__device__ __forceinline__ void pair_add(float& S, float& C, float p, float pe) {
  float s, e;
  two_sum(S, p, s, e);
  e += C + pe;
  S = s + e;
  C = e - (S - s);
}

}  // namespace ar
