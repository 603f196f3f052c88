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

// Dot-product operand split: (hi, lo) floats of a * 2^s, with the power of
// two s applied through the exponent field (exact).  Only the in-range case
// of d2f2 is built: 2^-74 <= |a 2^s| < 2^128 gives hi + lo = a 2^s to 2^-48
// relative; everything else (zero, smaller values, larger values, inf, nan)
// becomes (0, 0).  Callers keep the operands near 1 by their choice of s and
// test non-finite inputs separately.  sb = (128 + s) << 23 and
// lim = (949 - s) << 20 are per-column constants (two's complement, s in
// [-400, 400]).  Thirteen integer/FP32 operations, one of them on the
// conversion unit.
//   hb: the top 32 bits of a shifted left by 3 hold the low 8 exponent bits
//   and the leading 23 significand bits; adding (128 + s) << 23 turns the
//   low 8 bits of the double's exponent into the float's biased exponent
//   (e - 896 + s, valid whenever that lies in [1, 254]).
//   lo: the 29 remaining significand bits times 2^(E + s - 52), signed like a.
__device__ __forceinline__ F2 d2f2_dot(double a, uint32_t sb, uint32_t lim) {
  const uint32_t hi = (uint32_t)__double2hiint(a);
  const uint32_t lo = (uint32_t)__double2loint(a);
  const uint32_t t = __funnelshift_l(lo, hi, 3);
  const uint32_t hb = ((t + sb) & 0x7fffffffu) | (hi & 0x80000000u);
  const float sc = __uint_as_float((hb & 0xff800000u) - (52u << 23));
  const float tl = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), sc);
  const bool ok = ((hi & 0x7fffffffu) - lim) < (202u << 20);
  return ok ? F2{__uint_as_float(hb), tl} : F2{0.f, 0.f};
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

// Paired forms for two independent rows at once: Blackwell's FP32 pipe
// issues FADD2/FMUL2/FFMA2, two round-to-nearest float operations per
// instruction (one per component, each exactly as the scalar one), so the
// error-free transformations below cost half the issue slots of the scalar
// ones per row.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// a - b per component: the paired subtraction (PTX sub.rn.f32x2), so that
// no operand has to be negated first.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &t) {
  s = __fadd2_rn(a, b);
  const float2 bb = sub2(s, a);
  t = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// (S, C) += p + e per component (acc_add on two rows).
__device__ __forceinline__ void acc_add2(float2 &S, float2 &C, float2 p, float2 e) {
  float2 s, t;
  two_sum2(S, p, s, t);
  C = __fadd2_rn(C, __fadd2_rn(t, e));
  S = s;
}

// p + e = (h + l) * u per component: exact head product, tail to 2^-48.
__device__ __forceinline__ void prod_f2(float2 h, float2 l, float2 u, float2 &p, float2 &e) {
  p = __fmul2_rn(h, u);
  e = __ffma2_rn(h, u, neg2(p));
  e = __ffma2_rn(l, u, e);
}

// p + e = (ah + al) * (bh + bl) per component, to 2^-48 relative.
__device__ __forceinline__ void prod_ff2(float2 ah, float2 al, float2 bh, float2 bl, float2 &p,
                                         float2 &e) {
  p = __fmul2_rn(ah, bh);
  e = __ffma2_rn(ah, bh, neg2(p));
  e = __ffma2_rn(ah, bl, e);
  e = __ffma2_rn(al, bh, e);
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

// e^u for a double u on the FP32 pipe, table-driven (Tang's method:
// P. T. P. Tang, "Table-driven implementation of the exponential function
// in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989).
//   u = (128 q + j) ln2/128 + r,  |r| <= ln2/256,
//   e^u = 2^q * 2^(j/128) * e^r,
// with ln2/128 = L1 + L2 + L3 (L1 has 10 significant bits, so k L1 is exact
// for |k| < 2^14; L2, L3 are the next two float roundings), the table
// 2^(j/128) held as (hi, lo) float pairs, and
//   e^r = 1 + r + r^2/2 + r^3 (1/6 + r/24 + r^2/120),
// whose truncation error is below r^6/720 < 2^-59 and whose last group
// (below 2^-27) is evaluated in plain FP32.  Error: the split of u and the
// roundings in the reduced argument's low part carry an absolute error of up
// to about 3 |u| 2^-48, which becomes a relative error of e^u; the table and
// the (hi, lo) products add a few 2^-48: relative error <= 3 |u| 2^-48 +
// 2^-45.  Returns +inf above e^88.7 and 0 below e^-86.6.

constexpr int EXP_TAB = 128;

// Fills the table tab[j] = 2^(j/128) (one FP64 exp2 per entry, split
// exactly into two floats); call from every thread of the block, then
// synchronise before the first exp_df.
__device__ __forceinline__ void exp_table_init(float2 *tab) {
  for (int j = threadIdx.x; j < EXP_TAB; j += blockDim.x) {
    const F2 t = d2f2(exp2((double)j / (double)EXP_TAB));
    tab[j] = make_float2(t.h, t.l);
  }
}

__device__ __forceinline__ double exp_df(double u, const float2 *tab) {
  const float L1 = 0x1.628p-8f, L2 = 0x1.90bfbep-18f, L3 = 0x1.1cf79ap-43f;
  const float INV = 0x1.715476p+7f;  // 128 / ln2 rounded to float
  const F2 x = d2f2(u);
  const float kf = rintf(__fmul_rn(x.h, INV));
  if (kf > 16383.f) return __longlong_as_double(0x7ff0000000000000LL);
  if (kf < -16000.f) return 0.0;
  const int k = (int)kf;
  const float r0 = __fmaf_rn(-kf, L1, x.h);  // exact
  const float p = __fmul_rn(kf, L2), pe = __fmaf_rn(kf, L2, -p);
  float s, t;
  two_sum(r0, -p, s, t);
  const float low = __fadd_rn(__fsub_rn(t, pe), __fsub_rn(x.l, __fmul_rn(kf, L3)));
  const F2 r = fast_two_sum(s, low);
  // r^3 (1/6 + r/24 + r^2/120) in FP32
  const float c3 = __fmul_rn(__fmul_rn(r.h, __fmul_rn(r.h, r.h)),
                             __fmaf_rn(r.h, __fmaf_rn(r.h, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f));
  float q2, q2e;
  prod_ff(r, r, q2, q2e);
  F2 S = df_add(r, F2{__fmul_rn(0.5f, q2), __fmul_rn(0.5f, q2e)});  // r + r^2/2
  S = fast_two_sum(S.h, __fadd_rn(S.l, c3));
  F2 E = fast_two_sum(1.f, S.h);  // |S| < 2^-8
  E = fast_two_sum(E.h, __fadd_rn(E.l, S.l));
  const float2 T = tab[k & (EXP_TAB - 1)];
  float ph, pl;
  prod_ff(F2{T.x, T.y}, E, ph, pl);
  const F2 P = fast_two_sum(ph, pl);
  // P is in [0.99, 2): join it in FP64, then scale by 2^q through the
  // exponent field (exact; the result is a normal double for every q here)
  const double d = f2d(P.h) + f2d(P.l);
  return __hiloint2double(__double2hiint(d) + ((k >> 7) << 20), __double2loint(d));
}

}  // namespace aa
