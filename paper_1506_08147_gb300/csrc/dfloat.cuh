// Double-float arithmetic: a value is an unevaluated sum h + l of two FP32
// numbers with |l| <= ulp(h) / 2, about 48 significant bits.
//
// The error-free transformations are Knuth's two-sum, Dekker's fast
// two-sum and the FMA form of the exact product (a b = p + fma(a, b, -p)).
// Every product that feeds a sum is written with __fmul_rn so that the
// compiler never contracts it into an FMA, which would break the
// transformations.  The additions are the "sloppy" form: the error of
// a + b is within a few 2^-48 (|a| + |b|), the model that the backward
// error analyses of Cholesky and Householder reductions assume.
#pragma once

#include "common.cuh"

namespace dgdft {

struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl dfl_of(float x) { return {x, 0.0f}; }

__device__ __forceinline__ dfl dfl_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double dfl_val(dfl a) { return (double)a.h + (double)a.l; }

// s + e with |s| >= |e| (or s == 0) into a normalised pair
__device__ __forceinline__ dfl dfl_fast(float s, float e) {
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ dfl dfl_neg(dfl a) { return {-a.h, -a.l}; }

__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
  const float s = __fadd_rn(a.h, b.h);
  const float v = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v));
  return dfl_fast(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ dfl dfl_sub(dfl a, dfl b) { return dfl_add(a, dfl_neg(b)); }

__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return dfl_fast(p, e);
}

// exact scaling by a power of two
__device__ __forceinline__ dfl dfl_scale2(dfl a, float p2) { return {a.h * p2, a.l * p2}; }

// c + a b
__device__ __forceinline__ dfl dfl_fma(dfl a, dfl b, dfl c) {
  const float p = __fmul_rn(a.h, b.h);
  float pe = fmaf(a.h, b.h, -p);
  pe = fmaf(a.h, b.l, fmaf(a.l, b.h, pe));
  const float s = __fadd_rn(c.h, p);
  const float v = __fsub_rn(s, c.h);
  const float e = __fadd_rn(__fsub_rn(c.h, __fsub_rn(s, v)), __fsub_rn(p, v));
  return dfl_fast(s, __fadd_rn(e, __fadd_rn(pe, c.l)));
}

// c - a b
__device__ __forceinline__ dfl dfl_fnma(dfl a, dfl b, dfl c) { return dfl_fma(dfl_neg(a), b, c); }

// 1 / b: the FP32 reciprocal and one Newton step x + x (1 - b x), where the
// residual 1 - b x is formed exactly enough in double-float
__device__ __forceinline__ dfl dfl_rcp(dfl b) {
  const float x = __frcp_rn(b.h);
  const dfl r = dfl_fnma(b, dfl_of(x), dfl_of(1.0f));  // ~2^-24
  return dfl_fast(x, __fmul_rn(x, r.h));
}

// 1 / sqrt(a) for a > 0: the correctly rounded FP32 value and one Newton
// step y + y (1 - a y^2) / 2 with the residual formed in double-float
__device__ __forceinline__ dfl dfl_rsqrt(dfl a) {
  const float y = __frsqrt_rn(a.h);
  const float yy = __fmul_rn(y, y);
  const dfl y2 = {yy, fmaf(y, y, -yy)};
  const dfl r = dfl_fnma(a, y2, dfl_of(1.0f));  // ~2^-24
  return dfl_fast(y, __fmul_rn(0.5f * y, r.h));
}

__device__ __forceinline__ dfl dfl_abs(dfl a) { return a.h >= 0.0f ? a : dfl_neg(a); }

// sum over the warp; every lane gets lane 0's total (one summation order)
__device__ __forceinline__ dfl dfl_warp_sum(dfl v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const dfl w = {__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
    v = dfl_add(v, w);
  }
  return {__shfl_sync(0xffffffffu, v.h, 0), __shfl_sync(0xffffffffu, v.l, 0)};
}

// The same arithmetic as a scalar type with conversions and operators, for
// kernels templated on their arithmetic type (the FFT passes): converts from
// FP64 on construction and back to FP64 explicitly.
struct dff {
  float h, l;
  dff() = default;
  __host__ __device__ dff(double x) {
    h = (float)x;
    l = (float)(x - (double)h);
  }
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};
__device__ __forceinline__ dfl as_dfl(dff a) { return {a.h, a.l}; }
__device__ __forceinline__ dff as_dff(dfl a) {
  dff r;
  r.h = a.h;
  r.l = a.l;
  return r;
}
__device__ __forceinline__ dff operator+(dff a, dff b) { return as_dff(dfl_add(as_dfl(a), as_dfl(b))); }
__device__ __forceinline__ dff operator-(dff a, dff b) { return as_dff(dfl_sub(as_dfl(a), as_dfl(b))); }
__device__ __forceinline__ dff operator*(dff a, dff b) { return as_dff(dfl_mul(as_dfl(a), as_dfl(b))); }
__device__ __forceinline__ dff operator-(dff a) { return as_dff(dfl_neg(as_dfl(a))); }
__device__ __forceinline__ dff& operator+=(dff& a, dff b) { return a = a + b; }
__device__ __forceinline__ dff& operator-=(dff& a, dff b) { return a = a - b; }
__device__ __forceinline__ dff& operator*=(dff& a, dff b) { return a = a * b; }

// complex double-float: the same 16 bytes as double2
struct __align__(16) dffc {
  dff x, y;
};
template <> struct cplx_of<dff> { using type = dffc; };

}  // namespace dgdft
