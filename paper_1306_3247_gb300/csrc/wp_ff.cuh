// Float-float ("FP32 pair") real type for the complex128-accuracy form on GB300.
//
// GB300 executes FP64 at about 1/58 of its FP32 rate (measured: 1.2 vs 70 TFLOP/s), so a
// 256^3 FP64 step is bound by the FP64 pipe. A value here is the unevaluated sum hi + lo
// of two floats (|lo| <= ulp(hi)/2), about 48 significant bits. Sums use Knuth's
// two-sum of the high parts plus the low parts and one renormalisation; products use
// Dekker's exact product through an FMA (error-free transformations, Dekker 1971, Knuth
// TAOCP vol. 2). The rounded intrinsics keep nvcc from contracting or reordering the steps.
// A complex element is 16 bytes, the same HBM traffic as complex128.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace wp {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ explicit ff(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ ff ff_make(float h, float l) {
  ff r;
  r.hi = h;
  r.lo = l;
  return r;
}

// s + e -> normalised pair, assuming |s| >= |e| or s == 0
__device__ __forceinline__ ff ff_fast_renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return ff_make(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_fast_renorm(s, e);
}

// Sum without the final renormalisation: s = fl(a.hi + b.hi) and the exact error of that
// sum plus the low parts, left as an unnormalised pair (|lo| a few ulp of hi). Inside a
// butterfly, whose adds feed only further adds and the final renormalisation (ff_norm),
// this keeps the same precision and drops three operations per sum.
__device__ __forceinline__ ff ff_add_raw(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return ff_make(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_norm(ff a) { return ff_fast_renorm(a.hi, a.lo); }

__device__ __forceinline__ ff operator-(ff a) { return ff_make(-a.hi, -a.lo); }

__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ff_fast_renorm(p, e);
}

__device__ __forceinline__ ff& operator*=(ff& a, ff b) {
  a = a * b;
  return a;
}

// a.hi*b.hi - c.hi*d.hi + (cross terms), the real part of a complex product, with the
// two high products and their difference formed error-free before one renormalisation.
__device__ __forceinline__ ff ff_dot2(ff a, ff b, ff c, ff d, float sign_c) {
  const float ch = sign_c * c.hi, cl = sign_c * c.lo;
  const float p = __fmul_rn(a.hi, b.hi), q = __fmul_rn(ch, d.hi);
  const float ep = fmaf(a.hi, b.hi, -p), eq = fmaf(ch, d.hi, -q);
  const float s = __fadd_rn(p, q);
  const float bb = __fsub_rn(s, p);
  const float es = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(q, bb));
  float e = __fadd_rn(__fadd_rn(ep, eq), es);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(ch, d.lo, fmaf(cl, d.hi, e))));
  return ff_fast_renorm(s, e);
}

}  // namespace wp
