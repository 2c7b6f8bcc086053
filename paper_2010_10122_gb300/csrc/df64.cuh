// Double-float ("df64") arithmetic on the FP32 pipes: a value is the unevaluated sum hi + lo of
// two floats (48-bit significand).  Sums use the two-sum and products the fma-based two-product
// error-free transformations (Knuth; Dekker), each result renormalised to a pair with
// |lo| <= ulp(hi) / 2.  GB300 runs FP32 FMAs at 64x its FP64 rate, so a double-float operation
// of 4 to 15 FP32 instructions is several times cheaper than the FP64 one.
#pragma once
#include <cuda_runtime.h>

namespace wg {

struct dd {
  float h, l;
};
struct cdd {
  dd r, i;
};

__device__ __forceinline__ dd dd_make(float h, float l) { dd x; x.h = h; x.l = l; return x; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dd two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd_make(s, e);
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return dd_make(s, e);
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.h, b.h);
  float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return fast_two_sum(s.h, e);
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd_make(-a.h, -a.l); }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ cdd c_add(cdd a, cdd b) { cdd c; c.r = dd_add(a.r, b.r); c.i = dd_add(a.i, b.i); return c; }
__device__ __forceinline__ cdd c_sub(cdd a, cdd b) { cdd c; c.r = dd_sub(a.r, b.r); c.i = dd_sub(a.i, b.i); return c; }
// x.h y.h + u.h v.h (sign: su = +1 or -1 for the second product) with the cross terms, as one
// normalised pair: both leading products are split exactly (fma), summed exactly (two-sum),
// and the small terms (product errors, cross products, low parts) are accumulated in float.
// 19 FP32 operations instead of two products and a sum (25).
__device__ __forceinline__ dd dd_dot2(dd x, dd y, dd u, dd v, float su) {
  const float p1 = __fmul_rn(x.h, y.h);
  const float e1 = __fmaf_rn(x.h, y.h, -p1);
  const float uh = su * u.h, ul = su * u.l;
  const float p2 = __fmul_rn(uh, v.h);
  const float e2 = __fmaf_rn(uh, v.h, -p2);
  dd s = two_sum(p1, p2);
  float t = __fadd_rn(__fadd_rn(e1, e2), s.l);
  t = __fmaf_rn(x.h, y.l, t);
  t = __fmaf_rn(x.l, y.h, t);
  t = __fmaf_rn(uh, v.l, t);
  t = __fmaf_rn(ul, v.h, t);
  return fast_two_sum(s.h, t);
}
__device__ __forceinline__ cdd c_mul(cdd a, cdd b) {
  cdd c;
  c.r = dd_dot2(a.r, b.r, a.i, b.i, -1.0f);
  c.i = dd_dot2(a.r, b.i, a.i, b.r, 1.0f);
  return c;
}
__device__ __forceinline__ cdd c_scale(cdd a, dd s) { cdd c; c.r = dd_mul(a.r, s); c.i = dd_mul(a.i, s); return c; }
// multiply by -i (fwd = true) or +i
__device__ __forceinline__ cdd c_mul_mi(cdd a, bool fwd) {
  cdd c;
  if (fwd) { c.r = a.i; c.i = dd_neg(a.r); }
  else { c.r = dd_neg(a.i); c.i = a.r; }
  return c;
}

__device__ __forceinline__ cdd load_cdd(const float4& v) {
  cdd c; c.r = dd_make(v.x, v.y); c.i = dd_make(v.z, v.w); return c;
}
__device__ __forceinline__ float4 store_cdd(const cdd& c) { return make_float4(c.r.h, c.r.l, c.i.h, c.i.l); }

__device__ __forceinline__ dd split_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return dd_make(h, l);
}
__device__ __forceinline__ double join_double(dd x) { return (double)x.h + (double)x.l; }

// a * b + c, one rounding step of the pair arithmetic (product as in dd_mul, sum as in dd_add)
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const dd s = two_sum(c.h, p);
  const float t = __fadd_rn(s.l, __fadd_rn(c.l, e));
  return fast_two_sum(s.h, t);
}

}  // namespace wg
