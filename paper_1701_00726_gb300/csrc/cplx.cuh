// Minimal complex and SU(3)-matrix helpers for the device code.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace bri {

template <typename T> struct C {
  T re, im;
};

template <typename T> __host__ __device__ __forceinline__ C<T> cmk(T r, T i) { return C<T>{r, i}; }
template <typename T> __device__ __forceinline__ C<T> operator+(C<T> a, C<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ C<T> operator-(C<T> a, C<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __device__ __forceinline__ C<T> operator*(C<T> a, C<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __device__ __forceinline__ C<T> operator*(T s, C<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __device__ __forceinline__ C<T> conj(C<T> a) { return {a.re, -a.im}; }
// acc += a * b
template <typename T> __device__ __forceinline__ void cfma(C<T>& acc, C<T> a, C<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename T> __device__ __forceinline__ void cfma_cj(C<T>& acc, C<T> a, C<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

template <typename T> struct M3 {
  C<T> m[3][3];
};

template <typename T> __device__ __forceinline__ M3<T> mmul(const M3<T>& a, const M3<T>& b) {
  M3<T> r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C<T> s{0, 0};
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma(s, a.m[i][k], b.m[k][j]);
      r.m[i][j] = s;
    }
  return r;
}

template <typename T> __device__ __forceinline__ M3<T> adj(const M3<T>& a) {
  M3<T> r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a.m[j][i]);
  return r;
}

template <typename T> __device__ __forceinline__ void madd(M3<T>& a, const M3<T>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) a.m[i][j] = a.m[i][j] + b.m[i][j];
}

// ----------------------------------------------------------- storage conversions
__device__ __forceinline__ C<double> ld2(const double2* p) {
  double2 v = __ldg(p);
  return {v.x, v.y};
}
__device__ __forceinline__ C<float> ld2(const float2* p) {
  float2 v = __ldg(p);
  return {v.x, v.y};
}
__device__ __forceinline__ C<float> ld2(const __nv_bfloat162* p) {
  __nv_bfloat162 v = *p;
  float2 f = __bfloat1622float2(v);
  return {f.x, f.y};
}

}  // namespace bri
