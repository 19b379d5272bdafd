// Double-float arithmetic on the FP32 pipe: a value is a pair (hi, lo) of
// floats with hi + lo the represented number and |lo| <= ulp(hi) / 2, about
// 48 significant bits.  Products use the FMA error term, sums TwoSum (Knuth)
// or FastTwoSum (Dekker); every operation is spelled with a rounding
// intrinsic so the compiler contracts nothing.  Used where the GB300's FP64
// rate (about 1/64 of FP32) would otherwise bind the complex128 path.
#pragma once

namespace nufft {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_of(double x) {
  const float h = __double2float_rn(x);
  return DF{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.hi + (double)a.lo; }

// k[i] for a run-time i < N, by predicated moves over a register array
template <int N>
__device__ __forceinline__ DF df_pick(const DF* k, int i) {
  DF v = k[0];
#pragma unroll
  for (int t = 1; t < N; ++t)
    if (i == t) v = k[t];
  return v;
}

// ilogb(|x|) + 1 of a normal double from its exponent field; -1100 for zero, subnormals,
// infinities and NaN, which take no part in a tile's scale
__device__ __forceinline__ int df_bexp(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return (e == 0 || e == 0x7ff) ? -1100 : e - 1022;
}

// x 2^-sh as a pair of floats using integer and FP32 operations only: hi the leading 24
// bits of the 53-bit significand (truncated, exact), lo the remaining 29 bits rounded to a
// float, so hi + lo = x 2^-sh to a relative 2^-47.  Zero and subnormal x give 0 (below any
// float once the tile's largest value is scaled to [0.5, 1)); infinities and NaN give NaN.
__device__ __forceinline__ DF df_split_scaled(double x, int sh) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return DF{0.0f, 0.0f};
  if (e == 0x7ff) return DF{__int_as_float(0x7fc00000), 0.0f};
  const unsigned long long m = ((unsigned long long)b & 0xfffffffffffffULL) | (1ULL << 52);
  const int E = e - 1023 - sh;  // x 2^-sh = +-m 2^(E - 52)
  float hi = ldexpf(__uint2float_rn((unsigned)(m >> 29)), E - 23);
  float lo = ldexpf(__uint2float_rn((unsigned)(m & ((1u << 29) - 1))), E - 52);
  if (b < 0) {
    hi = -hi;
    lo = -lo;
  }
  return DF{hi, lo};
}

// FastTwoSum: |a| >= |b|
__device__ __forceinline__ DF df_quick(float a, float b) {
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// TwoSum: any a, b
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}
__device__ __forceinline__ DF df_norm(DF a) { return df_quick(a.hi, a.lo); }

__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = df_two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_quick(s.hi, s.lo);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick(p, e);
}

// s += a * b, with s left unnormalised (callers normalise after a run of terms)
__device__ __forceinline__ void df_mac(DF& s, const DF a, const DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const DF t = df_two_sum(s.hi, p);
  s.hi = t.hi;
  s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, e));
}

// sqrt(a), a >= 0: the float root refined by one Newton step in double-float.  The correction
// (a - s0^2) / (2 s0) is about 2^-24 of the root, so an approximate division (relative error
// ~2^-22) leaves an absolute error near 2^-48 in the result, the size of the rounding of a's
// own double-float operations.
__device__ __forceinline__ DF df_sqrt(DF a) {
  if (!(a.hi > 0.0f)) return DF{0.0f, 0.0f};
  const float s0 = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(s0, s0);
  const float pe = __fmaf_rn(s0, s0, -p);
  // residual a - s0^2, exact in its leading part
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
  return df_quick(s0, __fdividef(r, __fmul_rn(2.0f, s0)));
}

// e^x for -87 <= x <= 0 (x normalised; 2^k stays a normal float), to ~2^-47.5 relative for
// x >= -60 (below, the low part of the result nears the float underflow; the kernels evaluate
// x >= -2 beta >= -74, where such values lie below 1e-26).  Reduction x = k ln 2 + r,
// |r| <= ln(2)/2 + 2^-20, with
// ln 2 = LN2_HI + LN2_MID + LN2_LO (16, 16 and 24 bits): for |k| < 2^7 the products k LN2_HI and
// k LN2_MID are exact, x.hi - k LN2_HI is exact (Sterbenz), and two exact sums (TwoSum) add
// x.lo and -k LN2_MID, so r is known to ~2^-50.  e^r by its Taylor series to degree 12
// (remainder below 2e-16): the terms of degree 8..12 (at most 5e-9) in float, which costs them
// no more than 2^-51, the terms of degree 0..7 by Horner steps in double-float, each adding the
// float pair of 1/j! to r times the running value with FastTwoSum (|1/j!| exceeds the product)
// and the result left unnormalised until the end.  Then the exact scaling by 2^k.  Relative
// error ~2^-47.5 (checked against 120-bit arithmetic with the float operations emulated
// exactly); about a third of the operations of the plain degree-13 double-float Horner scheme.
__device__ __forceinline__ DF df_exp_neg(DF x) {
  const float k = rintf(__fmul_rn(x.hi, 1.44269504088896340736f));
  const float LN2_HI = 0x1.62e4p-1f;
  const float LN2_MID = 0x1.7f7ep-20f;
  const float LN2_LO = -1.2905320041778356e-11f;
  const float a = __fmaf_rn(-k, LN2_HI, x.hi);  // exact
  const DF s1 = df_two_sum(a, x.lo);
  const DF s2 = df_two_sum(s1.hi, -__fmul_rn(k, LN2_MID));  // k LN2_MID exact
  const DF r = df_quick(s2.hi, __fadd_rn(__fadd_rn(s1.lo, s2.lo), __fmul_rn(-k, LN2_LO)));
  // 1/j! for j = 0..7 as float pairs (hi, lo); j = 8..12 as floats
  const float fh[8] = {1.0f, 1.0f, 0.5f, 1.666666716e-01f, 4.166666791e-02f, 8.333333768e-03f, 1.388888923e-03f,
                       1.984127011e-04f};
  const float fl[8] = {0.0f, 0.0f, 0.0f, -4.967053879e-09f, -1.241763470e-09f, -4.346172033e-10f,
                       -3.363109444e-11f, -2.725596875e-12f};
  float t = 2.087675588e-09f;  // 1/12!
  t = __fmaf_rn(t, r.hi, 2.505210794e-08f);
  t = __fmaf_rn(t, r.hi, 2.755731998e-07f);
  t = __fmaf_rn(t, r.hi, 2.755731884e-06f);
  t = __fmaf_rn(t, r.hi, 2.480158764e-05f);
  DF y = {t, 0.0f};
#pragma unroll
  for (int j = 7; j >= 0; --j) {
    const float p = __fmul_rn(r.hi, y.hi);
    float e = __fmaf_rn(r.hi, y.hi, -p);
    e = __fmaf_rn(r.hi, y.lo, e);
    e = __fmaf_rn(r.lo, y.hi, e);
    const float sh = __fadd_rn(fh[j], p);
    const float err = __fsub_rn(p, __fsub_rn(sh, fh[j]));
    y = DF{sh, __fadd_rn(err, __fadd_rn(e, fl[j]))};
  }
  y = df_norm(y);
  const float sc = __int_as_float(((int)k + 127) << 23);  // 2^k, normal for k >= -126
  return DF{__fmul_rn(y.hi, sc), __fmul_rn(y.lo, sc)};
}

// The ES kernel (Eq. (ES)) exp(beta (sqrt(1 - z^2) - 1)) in double-float; with cosh_kernel
// its smooth variant (Remark in Sec. 7) as e^{beta (s - 1)} + e^{-beta (s + 1)}, both
// exponents in [-2 beta, 0].
__device__ __forceinline__ DF es_eval_df_z(DF z, DF beta, int cosh_kernel = 0) {
  const DF z2 = df_mul(z, z);
  const DF a = df_add(DF{1.0f, 0.0f}, DF{-z2.hi, -z2.lo});
  const DF s = df_sqrt(a);
  const DF x = df_mul(beta, df_add(s, DF{-1.0f, 0.0f}));
  if (!cosh_kernel) return df_exp_neg(x);
  const DF x2 = df_mul(beta, df_add(s, DF{1.0f, 0.0f}));
  return df_add(df_exp_neg(x), df_exp_neg(DF{-x2.hi, -x2.lo}));
}
__device__ __forceinline__ DF es_eval_df(double z, DF beta, int cosh_kernel = 0) {
  return es_eval_df_z(df_of(z), beta, cosh_kernel);
}

}  // namespace nufft
