#pragma once
// aa_df.cuh -- arithmetic on the FP32 and integer pipes for values held as
// an unevaluated sum of two floats (hi + lo), with conversions to and from
// FP64 built from integer operations.
//
// Why: on GB300 the FP64 pipe retires 2 fused multiply-adds per clock per SM
// (measured 0.60 TFMA/s on the whole GPU) against 128 per clock on the FP32
// pipe, and the hardware float<->double conversions run on the FP64 pipe too.
// A pass that converts or multiplies FP64 data at HBM speed therefore has
// to do that work on the FP32/INT pipes.
//
// Methods (all exact, round-to-nearest FP32 operations; the explicit
// __f*_rn intrinsics keep the compiler from contracting a product into a
// following sum, which would break exactness):
//  - TwoSum: s + t = a + b exactly (Knuth, TAOCP vol. 2, 4.2.2);
//  - FastTwoSum: the same when |a| >= |b| (Dekker 1971);
//  - TwoProd: p + e = a * b exactly via one fused multiply-add (Ogita, Rump,
//    Oishi 2005, "Accurate sum and dot product").
// Splitting a double gives hi = its leading 24 significant bits and lo = the
// remaining 29 bits rounded to 24, so |a - (hi + lo)| <= 2^-48 |a| for
// 2^-74 <= |a| < 2^128 (below 2^-74 lo is dropped and the split has float
// precision; below 2^-126 both parts are zero).
#include <stdint.h>

namespace aa {

struct F2 {
  float h, l;
};

// float -> double, exact, integer operations only.  Subnormal floats become
// signed zero; infinities and NaNs keep their class.
__device__ __forceinline__ double f2d(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t s = b & 0x80000000u;
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t m = b & 0x7fffffu;
  uint32_t hi = s | ((e + 896u) << 20) | (m >> 3);
  const uint32_t lo = m << 29;
  hi = (e == 0u) ? s : hi;
  hi = (e == 0xffu) ? (s | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u)) : hi;
  return __hiloint2double((int)hi, (int)((e == 0u) ? 0u : lo));
}

// double -> (hi, lo) floats with hi + lo = a to 2^-48 relative; integer
// operations, one integer-to-float conversion and one multiply.
__device__ __forceinline__ F2 d2f2(double a) {
  const uint32_t hi = (uint32_t)__double2hiint(a);
  const uint32_t lo = (uint32_t)__double2loint(a);
  const uint32_t s = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int ef = e - 896;  // float biased exponent of the head
  uint32_t hb = s | ((uint32_t)(ef > 0 ? ef : 0) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t L = lo & 0x1fffffffu;  // tail significand: L * 2^(e - 1075)
  const int es = e - 948;                // biased float exponent of 2^(e - 1075)
  const float sc = __uint_as_float((uint32_t)(es > 0 ? es : 0) << 23);
  float tl = __fmul_rn(__uint2float_rn(L), sc);
  tl = s ? -tl : tl;
  if (ef <= 0) {  // |a| < 2^-126 (or zero): flush
    hb = s;
    tl = 0.f;
  }
  if (ef >= 255) {  // inf, nan, or beyond float range
    const bool nan = (e == 0x7ff) && (((hi & 0xfffffu) | lo) != 0u);
    hb = s | 0x7f800000u | (nan ? 0x400000u : 0u);
    tl = 0.f;
  }
  return F2{__uint_as_float(hb), tl};
}

// hi + lo -> double (one FP64 add; exact when the parts do not overlap).
__device__ __forceinline__ double f22d(F2 a) { return f2d(a.h) + f2d(a.l); }

// double -> float, round to nearest (exact except within 2^-47 of a tie).
__device__ __forceinline__ float d2f_rn(double a) {
  const F2 x = d2f2(a);
  return __fadd_rn(x.h, x.l);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = c * u (c = (c.h, c.l), u a float): exact head product, tail to 2^-48.
__device__ __forceinline__ void prod_f(F2 c, float u, float &p, float &e) {
  p = __fmul_rn(c.h, u);
  e = __fmaf_rn(c.h, u, -p);
  e = __fmaf_rn(c.l, u, e);
}

// p + e = a * b for two (hi, lo) pairs, to 2^-48 relative.
__device__ __forceinline__ void prod_ff(F2 a, F2 b, float &p, float &e) {
  p = __fmul_rn(a.h, b.h);
  e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
}

// (S, C) += p + e: compensated accumulation (TwoSum on the head).
__device__ __forceinline__ void acc_add(float &S, float &C, float p, float e) {
  float s, t;
  two_sum(S, p, s, t);
  C = __fadd_rn(C, __fadd_rn(t, e));
  S = s;
}

// a + c * u for a (hi, lo) accumulator a, constant c and float u; normalised.
__device__ __forceinline__ F2 df_axpy_f(F2 a, F2 c, float u) {
  float p, e, s, t;
  prod_f(c, u, p, e);
  two_sum(a.h, p, s, t);
  t = __fadd_rn(t, __fadd_rn(a.l, e));
  return fast_two_sum(s, t);
}

// u + c * a for a float u, constant c and (hi, lo) a; normalised.
__device__ __forceinline__ F2 df_axpy_ff(float u, F2 c, F2 a) {
  float p, e, s, t;
  prod_ff(c, a, p, e);
  two_sum(u, p, s, t);
  t = __fadd_rn(t, e);
  return fast_two_sum(s, t);
}

// (a + b) for two (hi, lo) pairs, normalised.
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
  float s, t;
  two_sum(a.h, b.h, s, t);
  t = __fadd_rn(t, __fadd_rn(a.l, b.l));
  return fast_two_sum(s, t);
}

// c * a + b for (hi, lo) pairs (one Horner step), normalised.
__device__ __forceinline__ F2 df_mad(F2 c, F2 a, F2 b) {
  float p, e, s, t;
  prod_ff(c, a, p, e);
  two_sum(b.h, p, s, t);
  t = __fadd_rn(t, __fadd_rn(b.l, e));
  return fast_two_sum(s, t);
}

// e^u for a double u on the FP32 pipe.  The split of u and the roundings in
// the reduced argument's low part carry an absolute error of up to about
// 3 |u| 2^-48, which becomes a relative error of e^u; the polynomial and the
// final scaling add a few 2^-48: relative error <= 3 |u| 2^-48 + 2^-45.
// Range reduction u = k ln2 + r with |r| <= ln2/2, ln2 = L1 + L2 + L3 (L1
// has a short significand, so k L1 is exact for |k| < 128); then
// e^r = sum_{j=0}^{13} r^j / j! by Horner's rule in (hi, lo) arithmetic
// (truncation error below 0.35^14/14! < 2^-52); finally the exact scaling by
// 2^k.  Returns +inf above the float range, 0 below it.
__device__ __forceinline__ double exp_df(double u) {
  // 1/j!, j = 0..13, as (hi, lo) float pairs (hi = 1/j! rounded to float,
  // lo = the rounded remainder)
  const float C[14][2] = {{1.0f, 0.0f},
                          {1.0f, 0.0f},
                          {0.5f, 0.0f},
                          {0.1666666716337204f, -4.967053879312289e-09f},
                          {0.0416666679084301f, -1.2417634698280722e-09f},
                          {0.008333333767950535f, -4.34617203337595e-10f},
                          {0.0013888889225199819f, -3.3631094437103215e-11f},
                          {0.00019841270113829523f, -2.725596874933456e-12f},
                          {2.4801587642286904e-05f, -3.40699609366682e-13f},
                          {2.7557318844628753e-06f, 3.793571224297229e-14f},
                          {2.755731998149713e-07f, -7.575112209051195e-15f},
                          {2.5052107943679403e-08f, 4.4176230446483665e-16f},
                          {2.0876755879584152e-09f, 1.1082839147459852e-16f},
                          {1.6059044372074283e-10f, -5.352526511562726e-18f}};
  const float L1 = 0x1.62e4p-1f, L2 = 0x1.7f7d1cp-20f, L3 = 0x1.ef357ap-45f;
  const F2 x = d2f2(u);
  const float kf = rintf(__fmul_rn(x.h, 1.44269502f));
  if (kf > 127.f) return __longlong_as_double(0x7ff0000000000000LL);
  if (kf < -125.f) return 0.0;
  const float r0 = __fmaf_rn(-kf, L1, x.h);  // exact
  const float p = __fmul_rn(kf, L2), pe = __fmaf_rn(kf, L2, -p);
  float s, t;
  two_sum(r0, -p, s, t);
  const float low = __fadd_rn(__fsub_rn(t, pe), __fsub_rn(x.l, __fmul_rn(kf, L3)));
  const F2 r = fast_two_sum(s, low);
  F2 P{C[13][0], C[13][1]};
#pragma unroll
  for (int j = 12; j >= 0; --j) P = df_mad(P, r, F2{C[j][0], C[j][1]});
  const float sc = __int_as_float(((int)kf + 127) << 23);
  return f2d(__fmul_rn(P.h, sc)) + f2d(__fmul_rn(P.l, sc));
}

}  // namespace aa
