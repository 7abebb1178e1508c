// Common device helpers: complex arithmetic on float2/double2, float-float
// ("double-single") arithmetic for the Stolt positions, launch checks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace isam {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) {
  cplx<T> r; r.x = re; r.y = im; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
// FP32: one packed two-lane instruction on sm_100 and later, each lane rounded
// to nearest like the scalar form (so the results are the same bits)
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fadd2_rn(a, b);
#else
  a.x += b.x; a.y += b.y; return a;
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
#else
  a.x -= b.x; a.y -= b.y; return a;
#endif
}
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
// FP32 product and scaling as packed two-lane multiplies / FMAs
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  const float2 p = __fmul2_rn(a, make_float2(b.x, b.x));                // (a.x b.x, a.y b.x)
  return __ffma2_rn(make_float2(-a.y, a.x), make_float2(b.y, b.y), p);
#else
  float2 r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
#endif
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fmul2_rn(a, make_float2(s, s));
#else
  a.x *= s; a.y *= s; return a;
#endif
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// acc + c y for a real c
template <typename C, typename T> __device__ __forceinline__ C cfma_r(T c, C y, C acc) {
  acc.x = fma(c, y.x, acc.x); acc.y = fma(c, y.y, acc.y); return acc;
}
__device__ __forceinline__ float2 cfma_r(float c, float2 y, float2 acc) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __ffma2_rn(make_float2(c, c), y, acc);
#else
  acc.x = fmaf(c, y.x, acc.x); acc.y = fmaf(c, y.y, acc.y); return acc;
#endif
}
// multiply by sign * i   (sign = +1 or -1)
template <int SIGN, typename C> __host__ __device__ __forceinline__ C cmul_i(C a) {
  C r; r.x = -SIGN * a.y; r.y = SIGN * a.x; return r;
}

// ---------------------------------------------------------------------------
// float-float arithmetic (Dekker / Knuth error-free transformations).  A value
// is hi + lo with |lo| <= ulp(hi)/2; about 44 bits of significand.
// ---------------------------------------------------------------------------
struct ff { float hi, lo; };

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff ff_quick(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  ff t = ff_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = ff_quick(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return ff_quick(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = ff_two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return ff_quick(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = ff_two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return ff_quick(p.hi, p.lo);
}
// float-float square root from an approximate seed r ~ sqrt(a.hi) (a few ulp):
// one Newton correction d = (a - r^2) / (2r), with r^2 formed exactly by an FMA
// and the division by an approximate reciprocal, gives ~44 significant bits.
__device__ __forceinline__ ff ff_sqrt_fast(ff a) {  // a > 0
  const float r = a.hi * rsqrtf(a.hi);
  const float e = __fadd_rn(__fmaf_rn(-r, r, a.hi), a.lo);
  return ff_quick(r, __fdividef(e, 2.0f * r));
}

}  // namespace isam
