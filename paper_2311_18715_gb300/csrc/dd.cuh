// Double-float ("dd") arithmetic on the FP32 pipes: a value is the unevaluated sum h + l
// of two floats with |l| <= ulp(h)/2, a 48-bit significand.  GB300 issues an FP32 FMA per
// warp every cycle but an FP64 one every 64 cycles (an FP64 division costs ~600), so the
// small solves of the update and the eigensolver run in this format.
//
// The error-free transformations are Knuth's two-sum, Dekker's fast-two-sum (|a| >= |b|)
// and the FMA-based two-product; products and sums are then renormalised.  Division takes
// two quotient digits, square root one Newton correction.  Every step uses explicitly
// rounded intrinsics so that no multiply-add is contracted behind our back.
#pragma once
#include <cuda_runtime.h>

#include "pair2d.cuh"

namespace odmd {

struct dd {
  float h, l;
};

__device__ __forceinline__ dd dd_of(float h) { return dd{h, 0.f}; }
__device__ __forceinline__ dd dd_of(float2 v) { return dd{v.x, v.y}; }
__device__ __forceinline__ float2 f2_of(dd a) { return make_float2(a.h, a.l); }
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.h + (double)a.l; }
// a double as the pair h = RN(x), l = RN(x - h): from x's bits by integer operations
// (pair2d.cuh; conversions and subtractions run at the FP64 rate), by conversions when a
// part falls outside the normal float range
__device__ __forceinline__ dd dd_from_double(double x) {
  dd r;
  if (!double_to_pair_fast(x, r.h, r.l)) {
    r.h = __double2float_rn(x);
    r.l = __double2float_rn(x - (double)r.h);
  }
  return r;
}
// a float pair (hi, lo) as the double it represents exactly, and a double rounded to a pair
__device__ __forceinline__ double dd2d(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ float2 d2f2(double x) {
  const dd r = dd_from_double(x);
  return make_float2(r.h, r.l);
}

__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dd two_sum_dd(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return dd{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
  const dd s = two_sum_dd(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dd operator-(dd a) { return dd{-a.h, -a.l}; }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dd operator*(dd a, float b) {
  const float p = __fmul_rn(a.h, b);
  const float e = __fmaf_rn(a.l, b, __fmaf_rn(a.h, b, -p));
  return fast_two_sum(p, e);
}

// a*b + c with one renormalisation
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const dd s = two_sum_dd(p, c.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(e, c.l)));
}

__device__ __forceinline__ dd dd_div(dd a, dd b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  if (!isfinite(q1)) return dd{q1, 0.f};  // overflow or 0/0: no correction terms
  const dd r = a - b * q1;
  const float q2 = __fdiv_rn(r.h, b.h);
  const dd r2 = r - b * q2;
  const float q3 = __fdiv_rn(r2.h, b.h);
  const dd q = fast_two_sum(q1, q2);
  return q + dd_of(q3);
}

__device__ __forceinline__ dd dd_sqrt(dd a) {
  if (!(a.h > 0.f)) return dd{0.f, 0.f};
  const float s = __fsqrt_rn(a.h);
  const float p = __fmul_rn(s, s);
  const float pe = __fmaf_rn(s, s, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), pe), a.l);
  return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}

__device__ __forceinline__ dd dd_abs(dd a) { return a.h < 0.f || (a.h == 0.f && a.l < 0.f) ? -a : a; }
__device__ __forceinline__ bool dd_lt(dd a, dd b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ bool dd_gt(dd a, dd b) { return dd_lt(b, a); }
__device__ __forceinline__ bool dd_le(dd a, dd b) { return !dd_lt(b, a); }
__device__ __forceinline__ dd dd_max(dd a, dd b) { return dd_lt(a, b) ? b : a; }
__device__ __forceinline__ dd dd_min(dd a, dd b) { return dd_lt(a, b) ? a : b; }
__device__ __forceinline__ bool dd_isfinite(dd a) { return isfinite(a.h) && isfinite(a.l); }
// exact scaling by a power of two
__device__ __forceinline__ dd dd_ldexp(dd a, int e) { return dd{ldexpf(a.h, e), ldexpf(a.l, e)}; }

__device__ __forceinline__ dd dd_shfl_xor(dd a, int o) {
  return dd{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}
__device__ __forceinline__ dd dd_warp_sum(dd a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = a + dd_shfl_xor(a, o);
  return a;
}
__device__ __forceinline__ dd dd_warp_max(dd a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = dd_max(a, dd_shfl_xor(a, o));
  return a;
}

// complex double-float
struct cdd {
  dd re, im;
};
__device__ __forceinline__ cdd operator+(cdd a, cdd b) { return cdd{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cdd operator-(cdd a, cdd b) { return cdd{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cdd operator*(cdd a, cdd b) {
  return cdd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ dd cdd_abs2(cdd a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ cdd cdd_div(cdd a, cdd b) {
  // scale by the larger component of b (a power of two) to keep |b|^2 in range
  const float big = fmaxf(fabsf(b.re.h), fabsf(b.im.h));
  int e = 0;
  frexpf(big, &e);
  const cdd bs{dd_ldexp(b.re, -e), dd_ldexp(b.im, -e)};
  const cdd as{dd_ldexp(a.re, -e), dd_ldexp(a.im, -e)};
  const dd den = cdd_abs2(bs);
  const cdd num{as.re * bs.re + as.im * bs.im, as.im * bs.re - as.re * bs.im};
  return cdd{dd_div(num.re, den), dd_div(num.im, den)};
}

}  // namespace odmd
