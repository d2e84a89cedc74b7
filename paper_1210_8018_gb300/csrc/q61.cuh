// q61.cuh -- 64-bit fixed point with 61 fractional bits (Q61) for exact products of SU(3) matrices on the
// integer pipe (the handover transform of the mixed schedule and the large-step double update).
#pragma once
#include "su3.cuh"

namespace lgf {

// Products of SU(3) matrices in Q61 on the integer pipe, which on this GPU runs many times faster than the
// FP64 pipe. Every entry of an SU(3) matrix, of a product of two, and every partial sum formed here is at
// most 1 in magnitude (the partial sums are bounded by sum_k |a_k| |b_k| <= |a| |b| = 1 for unit rows and
// columns), so Q61 values stay near or below 2^61 and the integer sums never overflow. A product splits each factor into a signed high limb and a
// 31-bit low limb, so the three partial products it keeps are 32 x 32 -> 64-bit multiplies; the
// dropped low product and the truncation leave an error below 2^-59, and the result, rounded once to
// double, is exact to FP64 rounding.
__device__ __forceinline__ long long to_q61(double x) {  // x 2^61 toward zero, |x| < 2
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ed = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int sh = ed - 1014;  // x 2^61 = m 2^(ed - 1075 + 61)
  unsigned long long q = sh >= 0 ? m << (sh & 15) : (sh > -64 ? m >> (-sh) : 0ull);
  if (ed == 0) q = 0ull;
  return (long long)b < 0 ? -(long long)q : (long long)q;
}
__device__ __forceinline__ double from_q61(long long q) {  // q 2^-61, rounded to nearest (ties to even)
  if (q == 0) return 0.0;
  const unsigned long long sign = q < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long m = q < 0 ? (unsigned long long)(-q) : (unsigned long long)q;
  const int lz = __clzll((long long)m);
  m <<= lz;  // leading one at bit 63, of weight 2^(2 - lz)
  unsigned long long mant = m >> 11;
  const unsigned long long rest = m & 0x7FFull;
  if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ++mant;
  int e = 2 - lz;
  if (mant >> 53) {
    mant >>= 1;
    ++e;
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 1023) << 52) |
                                          (mant & 0x000FFFFFFFFFFFFFull)));
}
__device__ __forceinline__ long long mul_q61(long long a, long long b) {
  const int ah = (int)(a >> 31), bh = (int)(b >> 31);                       // |.| <= 2^30
  const int al = (int)(a & 0x7FFFFFFFll), bl = (int)(b & 0x7FFFFFFFll);     // [0, 2^31)
  const long long cross = (long long)ah * bl + (long long)al * bh;         // |.| < 2^62
  return (((long long)ah * bh) << 1) + (cross >> 30);
}
struct cq {
  long long r, i;
};
__device__ __forceinline__ cq to_cq(cx<double> v) { return {to_q61(v.r), to_q61(v.i)}; }
__device__ __forceinline__ void cq_mac(cq &acc, cq a, cq b) {  // acc += a b
  acc.r += mul_q61(a.r, b.r) - mul_q61(a.i, b.i);
  acc.i += mul_q61(a.r, b.i) + mul_q61(a.i, b.r);
}
__device__ __forceinline__ void cq_mac_cj(cq &acc, cq a, cq b) {  // acc += a conj(b)
  acc.r += mul_q61(a.r, b.r) + mul_q61(a.i, b.i);
  acc.i += mul_q61(a.i, b.r) - mul_q61(a.r, b.i);
}
__device__ __forceinline__ cq cq_cross_cj(cq a, cq b, cq c, cq d) {  // conj(a b - c d)
  cq t = {0, 0};
  cq_mac(t, a, b);
  cq_mac(t, {-c.r, -c.i}, d);
  return {t.r, -t.i};
}

}  // namespace lgf
