// Double-float complex arithmetic for the pivot blocks of the auxiliary
// matrix's separator fronts in the mixed form.
//
// A real number is held as the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, about 48 significant bits.  GB300 issues FP32
// arithmetic at about 64 times its FP64 rate, so a pivot block whose
// elimination is a chain of dependent columns runs several times faster in
// this form than in FP64, while its rounding (2^-48 relative to the
// operands) stays far below the FP32 rounding of the fronts around it.
//
// The building blocks are error-free transformations from the literature:
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   * Fast2Sum (Dekker 1971), for |a| >= |b|: s + e = a + b exactly;
//   * the FMA form of Dekker's product: p + e = a * b exactly with
//     e = fma(a, b, -p).
// Every step uses the explicitly rounded intrinsics (__fadd_rn, __fmul_rn,
// __fmaf_rn), which the compiler never contracts or reassociates, so the
// transformations stay exact.  Additions are the cheap ("sloppy") double-float
// sum: its error is at most about 2^-48 (|a| + |b|), an error relative to the
// operands, which is what the backward error of an elimination step needs.
// The reciprocal takes one Newton step from the FP32 reciprocal.
#pragma once
#include <cuda_runtime.h>

#include "dd_complex.cuh"

namespace ddk {

struct dfloat {
  float hi, lo;
};
// complex double-float, 16 bytes like double2
struct __align__(16) dfc {
  dfloat x, y;
};

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ dfloat df_neg(dfloat a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  dfloat r;
  df_fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
// the exact product a.hi * b.hi as p + e, plus the cross terms into e
__device__ __forceinline__ void df_prod(dfloat a, dfloat b, float& p, float& e) {
  p = __fmul_rn(a.hi, b.hi);
  e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  float p, e;
  df_prod(a, b, p, e);
  dfloat r;
  df_fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
// c - a * b
__device__ __forceinline__ dfloat df_fms(dfloat a, dfloat b, dfloat c) {
  float p, pe, s, e;
  df_prod(a, b, p, pe);
  df_two_sum(c.hi, -p, s, e);
  e = __fadd_rn(e, __fsub_rn(c.lo, pe));
  dfloat r;
  df_fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
// 1 / n: r0 = the FP32 reciprocal, then r = r0 + r0 (1 - n r0) (Newton)
__device__ __forceinline__ dfloat df_rcp(dfloat n) {
  const float r0 = __frcp_rn(n.hi);
  float e = __fmaf_rn(-n.hi, r0, 1.0f);
  e = __fmaf_rn(-n.lo, r0, e);
  dfloat r;
  df_fast_two_sum(r0, __fmul_rn(r0, e), r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dfc cmul(dfc a, dfc b) {
  dfc r;
  r.x = df_fms(a.y, b.y, df_mul(a.x, b.x));
  r.y = df_fms(df_neg(a.y), b.x, df_mul(a.x, b.y));
  return r;
}
// c - a * b
__device__ __forceinline__ dfc cfms(dfc a, dfc b, dfc c) {
  c.x = df_fms(df_neg(a.y), b.y, df_fms(a.x, b.x, c.x));
  c.y = df_fms(a.y, b.x, df_fms(a.x, b.y, c.y));
  return c;
}
// 1 / d (pivot magnitudes of these matrices are far from the limits of the
// FP32 exponent range, so |d|^2 cannot overflow)
__device__ __forceinline__ dfc crcp(dfc d) {
  const dfloat s = df_rcp(df_add(df_mul(d.x, d.x), df_mul(d.y, d.y)));
  dfc r;
  r.x = df_mul(d.x, s);
  r.y = df_mul(df_neg(d.y), s);
  return r;
}

template <> __device__ __forceinline__ dfc cconv<dfc, float2>(float2 a) {
  dfc r;
  r.x = {a.x, 0.f};
  r.y = {a.y, 0.f};
  return r;
}
// hi is the double-float value rounded to FP32 (|lo| <= ulp(hi) / 2)
template <> __device__ __forceinline__ float2 cconv<float2, dfc>(dfc a) { return make_float2(a.x.hi, a.y.hi); }
template <> __device__ __forceinline__ double2 cconv<double2, dfc>(dfc a) {
  return make_double2((double)a.x.hi + (double)a.x.lo, (double)a.y.hi + (double)a.y.lo);
}

}  // namespace ddk
