// Small complex helpers for interleaved double2 / float2 storage.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ddk {

template <typename S> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };

template <typename C> __device__ __forceinline__ C cmake(typename RealOf<C>::T x, typename RealOf<C>::T y) {
  C r; r.x = x; r.y = y; return r;
}
template <typename C> __device__ __forceinline__ C czero() { return cmake<C>(0, 0); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// c + a * b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
// c - a * b
template <typename C> __device__ __forceinline__ C cfms(C a, C b, C c) {
  c.x = fma(-a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
// a / b with the scaling of Smith (1962) to avoid overflow in |b|^2
template <typename C> __device__ __forceinline__ C cdiv(C a, C b) {
  using R = typename RealOf<C>::T;
  if (fabs(b.x) >= fabs(b.y)) {
    R r = b.y / b.x, den = b.x + b.y * r;
    return cmake<C>((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  } else {
    R r = b.x / b.y, den = b.x * r + b.y;
    return cmake<C>((a.x * r + a.y) / den, (a.y * r - a.x) / den);
  }
}
template <typename C> __device__ __forceinline__ double cabs2d(C a) {
  return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

template <typename D, typename S> __device__ __forceinline__ D cconv(S a) {
  return cmake<D>((typename RealOf<D>::T)a.x, (typename RealOf<D>::T)a.y);
}

}  // namespace ddk
