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

// sqrt(a), a >= 0: the float root refined by one Newton step in double-float
__device__ __forceinline__ DF df_sqrt(DF a) {
  if (!(a.hi > 0.0f)) return DF{0.0f, 0.0f};
  const float s0 = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(s0, s0);
  const float pe = __fmaf_rn(s0, s0, -p);
  // residual a - s0^2, exact in its leading part
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
  return df_quick(s0, __fdiv_rn(r, __fmul_rn(2.0f, s0)));
}

// e^x for x <= 0 (x >= -100): x = k ln 2 + r, |r| <= ln(2)/2, e^r by its Taylor
// series to degree 13 (remainder below 2e-16), then the exact scaling by 2^k.
__device__ __forceinline__ DF df_exp_neg(DF x) {
  const float k = rintf(__fmul_rn(x.hi, 1.44269504088896340736f));
  // ln 2 = LN2_HI + LN2_LO with LN2_HI holding 16 bits, so k * LN2_HI is exact for |k| < 2^8
  const float LN2_HI = 0.693145751953125f;
  const float LN2_LO = 1.42860682030941723212e-6f;
  DF r = df_add(x, DF{__fmul_rn(-k, LN2_HI), 0.0f});
  r = df_add(r, df_mul(DF{-k, 0.0f}, DF{LN2_LO, 0.0f}));
  // Horner with 1/j! for j = 13 .. 0, each as a pair of floats (hi, lo)
  const float fh[14] = {1.000000000e+00f, 1.000000000e+00f, 5.000000000e-01f, 1.666666716e-01f, 4.166666791e-02f,
                        8.333333768e-03f, 1.388888923e-03f, 1.984127011e-04f, 2.480158764e-05f, 2.755731884e-06f,
                        2.755731998e-07f, 2.505210794e-08f, 2.087675588e-09f, 1.605904437e-10f};
  const float fl[14] = {0.0f, 0.0f, 0.0f, -4.967053879e-09f, -1.241763470e-09f, -4.346172033e-10f,
                        -3.363109444e-11f, -2.725596875e-12f, -3.406996094e-13f, 3.793571224e-14f,
                        -7.575112209e-15f, 4.417623045e-16f, 1.108283981e-16f, -5.352526512e-18f};
  DF y = DF{fh[13], fl[13]};
#pragma unroll
  for (int j = 12; j >= 0; --j) y = df_add(df_mul(y, r), DF{fh[j], fl[j]});
  const int ki = (int)k;
  return DF{ldexpf(y.hi, ki), ldexpf(y.lo, ki)};
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
