// su3.cuh -- complex and 3x3 complex-matrix helpers for the gauge-fixing kernels (float or double).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df64.cuh"

namespace lgf {

template <typename T> struct cx {
  T r, i;
};

template <typename T> struct vec2;
template <> struct vec2<double> { using type = double2; };
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<df64> { using type = float4; };  // (re.hi, re.lo, im.hi, im.lo)

template <typename T> __device__ __forceinline__ cx<T> mkc(T r, T i) { return cx<T>{r, i}; }
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return {fma(a.r, b.r, -a.i * b.i), fma(a.r, b.i, a.i * b.r)};
}
template <typename T> __device__ __forceinline__ cx<T> scale(cx<T> a, T s) { return {a.r * s, a.i * s}; }
template <typename T> __device__ __forceinline__ cx<T> conjg(cx<T> a) { return {a.r, -a.i}; }
template <typename T> __device__ __forceinline__ T norm2(cx<T> a) { return fma(a.r, a.r, a.i * a.i); }
// acc + a*b
template <typename T> __device__ __forceinline__ cx<T> cmac(cx<T> acc, cx<T> a, cx<T> b) {
  acc.r = fma(a.r, b.r, acc.r);
  acc.r = fma(-a.i, b.i, acc.r);
  acc.i = fma(a.r, b.i, acc.i);
  acc.i = fma(a.i, b.r, acc.i);
  return acc;
}
// acc + a*conj(b)
template <typename T> __device__ __forceinline__ cx<T> cmac_cj(cx<T> acc, cx<T> a, cx<T> b) {
  acc.r = fma(a.r, b.r, acc.r);
  acc.r = fma(a.i, b.i, acc.r);
  acc.i = fma(a.i, b.r, acc.i);
  acc.i = fma(-a.r, b.i, acc.i);
  return acc;
}
// conj(a*b - c*d)
template <typename T> __device__ __forceinline__ cx<T> cross_cj(cx<T> a, cx<T> b, cx<T> c, cx<T> d) {
  cx<T> p = a * b, q = c * d;
  return {p.r - q.r, -(p.i - q.i)};
}

// Vector register form of one complex number, and back.
template <typename T> __device__ __forceinline__ cx<T> from_vec(typename vec2<T>::type v) { return {v.x, v.y}; }
template <> __device__ __forceinline__ cx<df64> from_vec<df64>(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
template <typename T> __device__ __forceinline__ typename vec2<T>::type to_vec(cx<T> a) {
  typename vec2<T>::type v;
  v.x = a.r;
  v.y = a.i;
  return v;
}
template <> __device__ __forceinline__ float4 to_vec<df64>(cx<df64> a) { return make_float4(a.r.hi, a.r.lo, a.i.hi, a.i.lo); }

// Read-only global load / store of one complex element (base counts real components of type T).
template <typename T> __device__ __forceinline__ cx<T> ldg(const T *base, int64_t idx) {
  return from_vec<T>(__ldg(reinterpret_cast<const typename vec2<T>::type *>(base) + idx));
}
template <typename T> __device__ __forceinline__ cx<T> ld(const T *base, int64_t idx) {
  return from_vec<T>(reinterpret_cast<const typename vec2<T>::type *>(base)[idx]);
}
template <typename T> __device__ __forceinline__ void st(T *base, int64_t idx, cx<T> a) {
  reinterpret_cast<typename vec2<T>::type *>(base)[idx] = to_vec<T>(a);
}

template <typename T> struct m3 {
  cx<T> e[9];
};

// c = a b
template <typename T> __device__ __forceinline__ void mul(const m3<T> &a, const m3<T> &b, m3<T> &c) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = a.e[3 * i] * b.e[j];
      acc = cmac(acc, a.e[3 * i + 1], b.e[3 + j]);
      acc = cmac(acc, a.e[3 * i + 2], b.e[6 + j]);
      c.e[3 * i + j] = acc;
    }
}
// c = a b^dagger
template <typename T> __device__ __forceinline__ void mul_adj(const m3<T> &a, const m3<T> &b, m3<T> &c) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = {0, 0};
      acc = cmac_cj(acc, a.e[3 * i], b.e[3 * j]);
      acc = cmac_cj(acc, a.e[3 * i + 1], b.e[3 * j + 1]);
      acc = cmac_cj(acc, a.e[3 * i + 2], b.e[3 * j + 2]);
      c.e[3 * i + j] = acc;
    }
}

// Rows 0 and 1 of c = a b (row 2 of c is left untouched).
template <typename T> __device__ __forceinline__ void mul_rows01(const m3<T> &a, const m3<T> &b, m3<T> &c) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = a.e[3 * i] * b.e[j];
      acc = cmac(acc, a.e[3 * i + 1], b.e[3 + j]);
      acc = cmac(acc, a.e[3 * i + 2], b.e[6 + j]);
      c.e[3 * i + j] = acc;
    }
}
// Rows 0 and 1 of c = a b^dagger.
template <typename T> __device__ __forceinline__ void mul_adj_rows01(const m3<T> &a, const m3<T> &b, m3<T> &c) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = {0, 0};
      acc = cmac_cj(acc, a.e[3 * i], b.e[3 * j]);
      acc = cmac_cj(acc, a.e[3 * i + 1], b.e[3 * j + 1]);
      acc = cmac_cj(acc, a.e[3 * i + 2], b.e[3 * j + 2]);
      c.e[3 * i + j] = acc;
    }
}
// Row 2 of an SU(3) matrix from rows 0 and 1: row2 = conj(row0 x row1).
template <typename T> __device__ __forceinline__ void complete_row2(m3<T> &m) {
  m.e[6] = cross_cj(m.e[1], m.e[5], m.e[2], m.e[4]);
  m.e[7] = cross_cj(m.e[2], m.e[3], m.e[0], m.e[5]);
  m.e[8] = cross_cj(m.e[0], m.e[4], m.e[1], m.e[3]);
}

// Projection to SU(3): normalise row 0; remove its component from row 1 and normalise;
// row 2 = conj(row0 x row1), which has determinant +1.
template <typename T> __device__ __forceinline__ void reunitarize(m3<T> &m) {
  T n0 = norm2(m.e[0]) + norm2(m.e[1]) + norm2(m.e[2]);
  T inv0 = rsqrt(n0);
#pragma unroll
  for (int j = 0; j < 3; ++j) m.e[j] = scale(m.e[j], inv0);
  cx<T> p = {0, 0};  // <r0, r1> = sum_j conj(r0_j) r1_j
#pragma unroll
  for (int j = 0; j < 3; ++j) p = cmac_cj(p, m.e[3 + j], m.e[j]);  // r1_j conj(r0_j)
#pragma unroll
  for (int j = 0; j < 3; ++j) m.e[3 + j] = m.e[3 + j] - p * m.e[j];
  T n1 = norm2(m.e[3]) + norm2(m.e[4]) + norm2(m.e[5]);
  T inv1 = rsqrt(n1);
#pragma unroll
  for (int j = 0; j < 3; ++j) m.e[3 + j] = scale(m.e[3 + j], inv1);
  m.e[6] = cross_cj(m.e[1], m.e[5], m.e[2], m.e[4]);
  m.e[7] = cross_cj(m.e[2], m.e[3], m.e[0], m.e[5]);
  m.e[8] = cross_cj(m.e[0], m.e[4], m.e[1], m.e[3]);
}

}  // namespace lgf
