// df64.cuh -- double-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is an unevaluated sum hi + lo of two float32 with |lo| <= ulp(hi)/2,
// carrying about 48 significant bits.  On this part the FP64 pipe issues
// 1/64 of the FP32 rate (measured 0.60 vs 37.2 TFMA/s, 71 vs 4.7 cycles of
// dependent latency), so hot loops that need float64-class results use this
// representation and keep float64 only at the interface.
//
// The building blocks are the classical error-free transformations:
//   two_sum       Knuth (TAOCP vol. 2, 4.2.2): s + e == a + b exactly;
//   fast_two_sum  Dekker (1971), requires |a| >= |b|;
//   two_prod      with a fused multiply-add: p + e == a * b exactly;
// and the double-word operations of Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM TOMS 44(2), 2017 ("sloppy" addition, multiplication with FMA, division
// by one Newton correction of the float quotient).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ehl {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df make_df(float h, float l) {
  df r;
  r.hi = h;
  r.lo = l;
  return r;
}

__device__ __forceinline__ df df_zero() { return make_df(0.f, 0.f); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df df_add(df x, df y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_neg(df x) { return make_df(-x.hi, -x.lo); }

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y) {
  float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_mul_f(df x, float y) {
  float p = __fmul_rn(x.hi, y);
  float e = __fmaf_rn(x.hi, y, -p);
  e = __fmaf_rn(x.lo, y, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// z - (a * b) - (c * d), one renormalisation at the end.
__device__ __forceinline__ df df_sub_two_prods(df z, df a, df b, df c, df d) {
  float p1 = __fmul_rn(a.hi, b.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  e1 = __fmaf_rn(a.hi, b.lo, e1);
  e1 = __fmaf_rn(a.lo, b.hi, e1);
  float p2 = __fmul_rn(c.hi, d.hi);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  e2 = __fmaf_rn(c.hi, d.lo, e2);
  e2 = __fmaf_rn(c.lo, d.hi, e2);
  float s, t, u;
  two_sum(z.hi, -p1, s, t);
  two_sum(s, -p2, s, u);
  float lo = __fadd_rn(__fadd_rn(z.lo, t), __fsub_rn(u, __fadd_rn(e1, e2)));
  df r;
  fast_two_sum(s, lo, r.hi, r.lo);
  return r;
}

// a * b - c * d
__device__ __forceinline__ df df_det2(df a, df b, df c, df d) {
  return df_sub_two_prods(df_mul(a, b), c, d, df_zero(), df_zero());
}

// x * y + z
__device__ __forceinline__ df df_fma(df x, df y, df z) {
  return df_sub_two_prods(z, df_neg(x), y, df_zero(), df_zero());
}

// 1 / y: float reciprocal refined by one Newton step in double-word.
__device__ __forceinline__ df df_rcp(df y) {
  float q = __frcp_rn(y.hi);
  // r = 1 - y * q  (computed in double-word), correction q * r
  df yq = df_mul_f(y, q);
  df r = df_sub(make_df(1.f, 0.f), yq);
  float c = __fmul_rn(q, r.hi);
  df out;
  fast_two_sum(q, c, out.hi, out.lo);
  return out;
}

__device__ __forceinline__ df df_div(df x, df y) {
  float q1 = __fdiv_rn(x.hi, y.hi);
  df r = df_sub(x, df_mul_f(y, q1));
  float q2 = __fdiv_rn(r.hi, y.hi);
  df out;
  fast_two_sum(q1, q2, out.hi, out.lo);
  return out;
}

__device__ __forceinline__ float df_abs_hi(df x) { return fabsf(x.hi); }

// float64 -> double-word without FP64 arithmetic: the 53-bit significand is
// cut into its leading 24 bits (hi, exact) and the remaining 29 bits (lo,
// rounded to 24 bits), using integer operations only.  Values whose
// magnitude is below 2^-100 are flushed to zero; +-Inf/NaN map to +-Inf/NaN
// in hi.  Relative representation error <= 2^-47.
__device__ __forceinline__ df df_from_double(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  unsigned hw = (unsigned)(b >> 32);
  unsigned lw = (unsigned)b;
  unsigned sign = hw & 0x80000000u;
  int e = (int)((hw >> 20) & 0x7ffu);
  df r;
  if (e >= 949 && e < 1151) {
    // |d| in [2^-74, 2^128): hi and the scale of lo are normal floats (one multiply, no branches)
    const int fe0 = e - 896;
    r.hi = __uint_as_float(sign | ((unsigned)fe0 << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    const float lo0 = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __uint_as_float((unsigned)(fe0 - 52) << 23));
    r.lo = __uint_as_float(__float_as_uint(lo0) | sign);
    return r;
  }
  if (e == 0x7ff) {  // Inf / NaN
    r.hi = __uint_as_float(sign | 0x7f800000u | (((hw & 0xfffffu) | lw) ? 0x400000u : 0u));
    r.lo = 0.f;
    return r;
  }
  int fe = e - 1023 + 127;  // float biased exponent of hi
  if (e == 0 || fe < 27) {  // zero, float64 subnormal or below 2^-100
    r.hi = __uint_as_float(sign);
    r.lo = 0.f;
    return r;
  }
  if (fe >= 255) {  // beyond float range
    r.hi = __uint_as_float(sign | 0x7f800000u);
    r.lo = 0.f;
    return r;
  }
  unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  r.hi = __uint_as_float(sign | ((unsigned)fe << 23) | m23);
  unsigned rest = lw & 0x1fffffffu;  // weight 2^(e - 1023 - 52)
  // rest * 2^(fe - 127 - 52): build the power of two (fe - 179 >= -152 here;
  // scale in two steps to stay inside the normal float range)
  float lo = __uint2float_rn(rest);
  int p = fe - 127 - 52;
  float s1 = __uint_as_float((unsigned)((p / 2) + 127) << 23);
  float s2 = __uint_as_float((unsigned)((p - p / 2) + 127) << 23);
  lo = __fmul_rn(__fmul_rn(lo, s1), s2);
  r.lo = sign ? -lo : lo;
  return r;
}

// The same split as df_from_double, bit for bit, without branches: every range's result is formed
// and the right one selected.  lo = rest * 2^p with p = fe - 179 scaled in two steps (both factors
// normal floats for p >= -152), which is the one multiply of the fast window whenever the product
// is normal.  For code whose throughput suffers from the branches (long straight-line kernels).
__device__ __forceinline__ df df_from_double_sel(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hw = (unsigned)(b >> 32);
  const unsigned lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  const int fe = e - 896;  // float biased exponent of hi
  const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const bool normal = (e >= 923) && (e < 1151);  // |d| in [2^-100, 2^128)
  const int p = normal ? fe - 179 : 0;
  const float s1 = __uint_as_float((unsigned)((p / 2) + 127) << 23);
  const float s2 = __uint_as_float((unsigned)((p - p / 2) + 127) << 23);
  const float lo = __fmul_rn(__fmul_rn(__uint2float_rn(lw & 0x1fffffffu), s1), s2);
  const unsigned big = sign | 0x7f800000u | ((e == 0x7ff && ((hw & 0xfffffu) | lw)) ? 0x400000u : 0u);
  df r;
  r.hi = __uint_as_float(normal ? (sign | ((unsigned)fe << 23) | m23) : (e >= 1151 ? big : sign));
  r.lo = normal ? __uint_as_float(__float_as_uint(lo) | sign) : 0.f;
  return r;
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

}  // namespace ehl
