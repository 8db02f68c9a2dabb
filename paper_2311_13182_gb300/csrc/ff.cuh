// Float-float ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// giving about 48 significant bits.  Sums and products are made exact with the
// error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the
// FMA-based exact product, following the double-double constructions of
// Hida, Li & Bailey (2001, "Algorithms for quad-double precision floating
// point arithmetic"), here one level down (float instead of double).
//
// Why: GB300 issues FP64 at a small fraction of its FP32 rate, and the path
// delays of the simulator need ~1e-9 relative precision (a 1e-4 relative
// IF-cube error allows ~6e-8 m of path length at 77 GHz).  Float-float gives
// ~1e-14 at roughly ten FP32 instructions per operation.
//
// The compiler must not reassociate these expressions; nvcc does not without
// fast-math flags, and every multiply-add that must stay fused is an explicit fmaf.
#pragma once

#include <math.h>

namespace sbr {

struct ff {
  float hi, lo;
};

__host__ __device__ inline ff ff_make(float hi, float lo) { return ff{hi, lo}; }
__host__ __device__ inline ff ff_of(float x) { return ff{x, 0.f}; }

// host: split a double into a normalised float pair
inline ff ff_from_double(double x) {
  const float hi = (float)x;
  return ff{hi, (float)(x - (double)hi)};
}

__device__ inline ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return ff{s, (a - (s - bb)) + (b - bb)};
}

__device__ inline ff fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  const float s = a + b;
  return ff{s, b - (s - a)};
}

__device__ inline ff two_prod(float a, float b) {
  const float p = a * b;
  return ff{p, fmaf(a, b, -p)};
}

// Sum with an error of a few units of 2^-44 relative to |a| + |b| (the
// "sloppy" double-double addition of Hida, Li & Bailey): exact sum of the hi
// parts, low parts added in FP32.  Under cancellation the result keeps that
// absolute accuracy, which is all the geometry here needs (~1e-13 of the
// operands' magnitude).
__device__ inline ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ inline ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ inline ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// exact difference of two floats as a float pair
__device__ inline ff ff_diff(float a, float b) { return two_sum(a, -b); }

__device__ inline ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, p.lo);
  p.lo = fmaf(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ inline ff ff_mulf(ff a, float b) {
  ff p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// long division: three float quotient digits
__device__ inline ff ff_div(ff a, ff b) {
  const float q1 = a.hi / b.hi;
  ff r = ff_sub(a, ff_mulf(b, q1));
  const float q2 = r.hi / b.hi;
  r = ff_sub(r, ff_mulf(b, q2));
  const float q3 = r.hi / b.hi;
  ff q = fast_two_sum(q1, q2);
  return ff_add(q, ff_of(q3));
}

// sqrt(a) = y + (a - y^2) / (2y) with y = sqrtf(hi): one Newton correction
__device__ inline ff ff_sqrt(ff a) {
  if (a.hi <= 0.f) return ff{0.f, 0.f};
  const float y = sqrtf(a.hi);
  const ff r = ff_sub(a, two_prod(y, y));
  return fast_two_sum(y, r.hi / (2.f * y));
}

// 1 / sqrt(a): float seed, one Newton step in float-float
__device__ inline ff ff_rsqrt(ff a) {
  const float y = rsqrtf(a.hi);
  // y' = y + y (1 - a y^2) / 2
  const ff ay2 = ff_mul(a, two_prod(y, y));
  const ff e = ff_sub(ff_of(1.f), ay2);
  return ff_add(ff_of(y), ff_mulf(e, 0.5f * y));
}

struct ff3 {
  ff x, y, z;
};

__device__ inline ff3 ff3_add(ff3 a, ff3 b) { return ff3{ff_add(a.x, b.x), ff_add(a.y, b.y), ff_add(a.z, b.z)}; }
__device__ inline ff3 ff3_sub(ff3 a, ff3 b) { return ff3{ff_sub(a.x, b.x), ff_sub(a.y, b.y), ff_sub(a.z, b.z)}; }
__device__ inline ff3 ff3_scale(ff3 a, ff s) { return ff3{ff_mul(a.x, s), ff_mul(a.y, s), ff_mul(a.z, s)}; }
__device__ inline ff ff3_dot(ff3 a, ff3 b) {
  return ff_add(ff_add(ff_mul(a.x, b.x), ff_mul(a.y, b.y)), ff_mul(a.z, b.z));
}
__device__ inline ff3 ff3_cross(ff3 a, ff3 b) {
  return ff3{ff_sub(ff_mul(a.y, b.z), ff_mul(a.z, b.y)), ff_sub(ff_mul(a.z, b.x), ff_mul(a.x, b.z)),
             ff_sub(ff_mul(a.x, b.y), ff_mul(a.y, b.x))};
}
// exact point difference of two float points
__device__ inline ff3 ff3_diff(float3 a, float3 b) { return ff3{ff_diff(a.x, b.x), ff_diff(a.y, b.y), ff_diff(a.z, b.z)}; }
__device__ inline ff3 ff3_of(float3 a) { return ff3{ff_of(a.x), ff_of(a.y), ff_of(a.z)}; }
__device__ inline float3 ff3_hi(ff3 a) { return make_float3(a.x.hi, a.y.hi, a.z.hi); }
__device__ inline ff ff3_len(ff3 a) { return ff_sqrt(ff3_dot(a, a)); }

}  // namespace sbr
