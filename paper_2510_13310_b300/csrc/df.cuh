// df.cuh -- double-float arithmetic: a value is an unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  Built from
// the error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2),
// FastTwoSum (Dekker 1971, |a| >= |b|) and the FMA form of TwoProduct; the
// addition is the accurate variant that renormalises twice (Hida, Li and Bailey,
// "Algorithms for quad-double precision floating point arithmetic", 2001).
//
// Every operation is spelled with round-to-nearest intrinsics so that the
// compiler neither contracts nor reorders the error terms.
#pragma once
#include <cuda_runtime.h>

namespace bab {

struct __align__(8) F2 {
  float h, l;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return F2{s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  F2 s = two_sum(a.h, b.h);
  const F2 t = two_sum(a.l, b.l);
  s = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}
__device__ __forceinline__ F2 f2_neg(F2 a) { return F2{-a.h, -a.l}; }
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) { return f2_add(a, f2_neg(b)); }
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
// a * b + c
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c) { return f2_add(f2_mul(a, b), c); }
// 1 / a: the FP32 reciprocal refined by one Newton step carried in double-float
// (the step's error is the square of the FP32 estimate's, ~2^-48)
__device__ __forceinline__ F2 f2_recip(F2 a) {
  const float y = __frcp_rn(a.h);
  float e = __fmaf_rn(-a.h, y, 1.0f);  // 1 - a.h y, exact
  e = __fmaf_rn(-a.l, y, e);
  return fast_two_sum(y, __fmul_rn(y, e));
}
// sqrt(a) for a > 0: FP32 square root refined by one Newton step in double-float
__device__ __forceinline__ F2 f2_sqrt(F2 a) {
  const float y = __fsqrt_rn(a.h);
  const F2 r = f2_sub(a, f2_mul(F2{y, 0.f}, F2{y, 0.f}));  // a - y^2, small
  return fast_two_sum(y, __fdiv_rn(r.h, __fmul_rn(2.0f, y)));
}
__device__ __forceinline__ bool f2_finite(F2 a) { return isfinite(a.h) && isfinite(a.l); }
__device__ __forceinline__ double f2_to_double(F2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ F2 f2_from_double(double x) {
  const float h = __double2float_rn(x);
  return F2{h, __double2float_rn(x - (double)h)};
}

}  // namespace bab
