// df64.cuh -- double-float ("df64") numbers: an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2),
// a 48-bit significand built from FP32 operations. On this GPU the FP64 pipe runs at 1/64 of the FP32
// rate, so the double-precision path does in df64 what does not need IEEE double:
//  * the Fourier filter: its error (~2^-47 relative to the norm of the field) is far below the 1e-12
//    agreement with the FP64 oracle, and the filter only sets the direction of the gauge update;
//  * the small-step forms of g and of the gauge update, which compute only the deviation of g from 1
//    (and the change of the link) in df64: that deviation is small, so its df64 error is at or below
//    the FP64 rounding of the result, which is assembled in FP64.
// Links, the theta/F sums and the general (large-step) forms stay in IEEE double.
//
// Building blocks (error-free transformations): TwoSum (Knuth), FastTwoSum (Dekker, |a| >= |b|) and
// TwoProd with a fused multiply-add; the double-word operations follow Joldes, Muller, Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word arithmetic" (2017):
// addition here is the "sloppy" variant (its error is bounded relative to |x| + |y|, which is the
// bound an FFT's normwise error analysis uses), multiplication is DWTimesDW.
#pragma once
#include <cuda_runtime.h>

namespace lgf {

struct df64 {
  float hi, lo;
};

__host__ __device__ constexpr df64 df64_from_double(double d) {
  return df64{(float)d, (float)(d - (double)(float)d)};
}
__device__ __forceinline__ double df64_to_double(df64 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df64 df64_from_double_rt(double d) {
  const float hi = __double2float_rn(d);
  return {hi, __double2float_rn(d - (double)hi)};
}

// (the _rn intrinsics keep the compiler from contracting or reassociating these exact steps)
__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
  const df64 s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df64 operator-(df64 x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }
__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
  const float tl1 = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo));
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}
// the double and float fma stay visible beside the df64 overload inside this namespace
using ::fma;
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
// x / y: a float quotient refined by one Newton step in df64.
__device__ __forceinline__ df64 operator/(df64 x, df64 y) {
  const float q1 = x.hi / y.hi;
  const df64 r = x - y * df64{q1, 0.f};
  const float q2 = r.hi / y.hi;
  return fast_two_sum(q1, q2);
}

// Constants and conversions for the arithmetic types float, double and df64.
template <typename T> __host__ __device__ constexpr T kconst(double c) { return (T)c; }
template <> __host__ __device__ constexpr df64 kconst<df64>(double c) { return df64_from_double(c); }

template <typename D, typename S> struct Conv {
  __device__ __forceinline__ static D f(S s) { return (D)s; }
};
// double -> df64 with integer operations only (the FP64 pipe is the scarce resource): hi takes the
// sign, the exponent and the top 23 stored mantissa bits (exact), lo the remaining 29 bits rounded to
// float and scaled; then the pair is renormalised. Magnitudes below 2^-126 (and zero) give 0, and a
// remainder below 2^-126 is dropped: both are far below the roundoff of the fields converted here.
__device__ __forceinline__ df64 df64_split_bits(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
  const int ed = (int)((hi32 >> 20) & 0x7FF);
  const int ef = ed - 1023 + 127;
  const unsigned sign = hi32 & 0x80000000u;
  if (ef < 1) return {0.f, 0.f};
  if (ef > 254) {  // beyond float range: infinity, or NaN kept as NaN (integer operations only)
    const bool nan = ed == 0x7FF && (((hi32 & 0xFFFFFu) | lo32) != 0);
    return {__uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u)), 0.f};
  }
  const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
  const int es = ed - 1075 + 127;  // exponent of 2^(e - 52) as a float
  float lo = 0.f;  // the truncated remainder has the sign of d
  if (es >= 1) {
    const float mag = (float)(lo32 & 0x1FFFFFFFu) * __uint_as_float((unsigned)es << 23);
    lo = sign ? -mag : mag;
  }
  return fast_two_sum(hi, lo);
}
// df64 -> double: each float is widened with integer operations (exact); one FP64 addition remains.
__device__ __forceinline__ double widen_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xFFu;
  if (ef == 0) return 0.0;  // zero (and float subnormals, far below the roundoff here)
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  ((unsigned long long)(ef == 0xFFu ? 0x7FFu : ef + 896u) << 52) |
                                  ((unsigned long long)(u & 0x7FFFFFu) << 29);  // Inf/NaN map to Inf/NaN
  return __longlong_as_double((long long)bits);
}
// double -> float, rounded to nearest (ties to even), with integer operations only. Results below the
// smallest normal float (2^-126) give a signed zero, results beyond the float range infinity (and NaN
// stays NaN): the fields converted here are O(1).
__device__ __forceinline__ float narrow_bits(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
  const unsigned sign = hi32 & 0x80000000u;
  const int ed = (int)((hi32 >> 20) & 0x7FF);
  const int ef = ed - 896;
  if (ed == 0x7FF) return __uint_as_float(sign | 0x7F800000u | ((((hi32 & 0xFFFFFu) | lo32) != 0) ? 0x400000u : 0u));
  if (ef < 1) return __uint_as_float(sign);
  if (ef > 254) return __uint_as_float(sign | 0x7F800000u);
  const unsigned m = ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29);  // top 23 stored mantissa bits
  const unsigned rest = lo32 & 0x1FFFFFFFu;                      // the 29 bits rounded away
  const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | ((((unsigned)ef << 23) | m) + up));  // a carry moves into the exponent
}
template <> struct Conv<df64, double> {
  __device__ __forceinline__ static df64 f(double s) { return df64_split_bits(s); }
};
template <> struct Conv<double, df64> {
  __device__ __forceinline__ static double f(df64 s) { return widen_bits(s.hi) + widen_bits(s.lo); }
};
template <> struct Conv<df64, df64> {
  __device__ __forceinline__ static df64 f(df64 s) { return s; }
};
template <> struct Conv<df64, float> {
  __device__ __forceinline__ static df64 f(float s) { return {s, 0.f}; }
};
template <typename D, typename S> __device__ __forceinline__ D convert(S s) { return Conv<D, S>::f(s); }

// double -> double-float without an integer-to-float conversion instruction: hi is the truncation to
// the top 24 significant bits (exact); the remaining 29 bits are rounded to 23 and placed in the
// mantissa field of a float whose implicit leading 1 is then subtracted (exact by Sterbenz's lemma; a
// carry out of the rounded field moves into the exponent, which gives the right value). The pair
// (hi, lo) is not renormalised: |lo| <= ulp(hi), and |hi + lo - d| <= 2^-47 |d|. Magnitudes below
// 2^-100 give 0 and the input must be finite; callers use it on matrix elements of magnitude <= 1.
__device__ __forceinline__ df64 df64_split_fast(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
  const int ed = (int)((hi32 >> 20) & 0x7FF);
  const unsigned sign = hi32 & 0x80000000u;
  const int ef = ed - 896;  // float exponent field of hi
  const int E = ed - 919;   // float exponent field whose mantissa unit is 2^(e - 46)
  if (E < 1) return {0.f, 0.f};
  const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
  const unsigned m = ((lo32 & 0x1FFFFFFFu) + 32u) >> 6;  // the remaining 29 bits rounded to 23 (may be 2^23)
  const unsigned base = sign | ((unsigned)E << 23);
  const float lo = __fsub_rn(__uint_as_float(base + m), __uint_as_float(base));
  return {hi, lo};
}

// Compensated accumulation of products of double-float numbers: the scheme of Ogita, Rump and Oishi,
// "Accurate sum and dot product" (2005, Dot2), applied to double-float operands. s collects the float
// sum of the leading products through TwoSum; c collects the exact product errors (FMA), the cross
// terms hi*lo and the TwoSum errors. The result s + c has an absolute error of a few 2^-48 times the
// sum of the magnitudes of the products.
struct dfacc {
  float s, c;
};
__device__ __forceinline__ dfacc dfacc_from(df64 x) { return {x.hi, x.lo}; }
// an accumulator holding the exact product x*y (to the dropped lo*lo term)
__device__ __forceinline__ dfacc dfacc_prod(df64 x, df64 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return {p, e};
}
__device__ __forceinline__ void dfacc_mac(dfacc &a, df64 x, df64 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const df64 t = two_sum(a.s, p);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
}
// the same with the product negated
__device__ __forceinline__ void dfacc_msub(dfacc &a, df64 x, df64 y) { dfacc_mac(a, df64{-x.hi, -x.lo}, y); }
__device__ __forceinline__ df64 dfacc_result(dfacc a) { return two_sum(a.s, a.c); }

}  // namespace lgf
