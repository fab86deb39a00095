// cos theta and sin theta as float-float pairs (about 48 bits, the precision of a complex64
// table record), with FP64 only in the argument reduction.
//
// GB300 issues FP64 instructions at 1/64 of its FP32 rate; an FP64 sincos per entry made
// the per-step potential tables of an uneven batch FP64 bound (ncu: FP64 pipe 37 % busy
// over the launch that forms them). Here FP64 does the reduction of the phase argument
// modulo pi/2 (Cody and Waite's reduction with pi/2 as the sum of two doubles):
// theta = q pi/2 + s, q = rint(2 theta / pi), |s| <= pi/4 up to rounding. sin s and cos s
// then come from their Taylor series, evaluated by Horner's rule in float-float
// arithmetic on the FP32 pipe (terms through s^17 and s^18: for |s| <= pi/4 the first
// omitted terms are below 2^-55 and 2^-57), and q mod 4 exchanges and negates the pair.
// Arguments beyond 2^20 in magnitude take the FP64 sincos.
#pragma once

#include <cuda_runtime.h>

#include "wp_ff.cuh"

namespace wp {

// 1/k! and its float-float parts, formed at compile time.
template <int K>
struct InvFact {
  static constexpr double v = InvFact<K - 1>::v / K;
  static constexpr float hi = (float)v;
  static constexpr float lo = (float)(v - (double)hi);
};
template <>
struct InvFact<0> {
  static constexpr double v = 1.0;
  static constexpr float hi = 1.0f;
  static constexpr float lo = 0.0f;
};

// 1/K! (NEG: -1/K!) as a float-float constant
template <int K, bool NEG>
__device__ __forceinline__ ff inv_fact_ff() {
  return NEG ? ff_make(-InvFact<K>::hi, -InvFact<K>::lo) : ff_make(InvFact<K>::hi, InvFact<K>::lo);
}

// sin s = s (1 - z/3! + z^2/5! - ... + z^8/17!), cos s = 1 - z/2! + ... + z^9/18!, z = s^2
__device__ __forceinline__ void sincos_taylor_ff(ff s, ff& sn, ff& cs) {
  const ff z = s * s;
  ff p = inv_fact_ff<17, false>();
  p = p * z + inv_fact_ff<15, true>();
  p = p * z + inv_fact_ff<13, false>();
  p = p * z + inv_fact_ff<11, true>();
  p = p * z + inv_fact_ff<9, false>();
  p = p * z + inv_fact_ff<7, true>();
  p = p * z + inv_fact_ff<5, false>();
  p = p * z + inv_fact_ff<3, true>();
  p = p * z + ff_make(1.0f, 0.0f);
  sn = s * p;
  ff c = inv_fact_ff<18, true>();
  c = c * z + inv_fact_ff<16, false>();
  c = c * z + inv_fact_ff<14, true>();
  c = c * z + inv_fact_ff<12, false>();
  c = c * z + inv_fact_ff<10, true>();
  c = c * z + inv_fact_ff<8, false>();
  c = c * z + inv_fact_ff<6, true>();
  c = c * z + inv_fact_ff<4, false>();
  c = c * z + inv_fact_ff<2, true>();
  cs = c * z + ff_make(1.0f, 0.0f);
}

// cos theta -> c, sin theta -> s
__device__ __forceinline__ void cis_ff(double theta, ff& c, ff& s) {
  if (!(fabs(theta) <= 1048576.0)) {
    double sd, cd;
    sincos(theta, &sd, &cd);
    c = ff(cd);
    s = ff(sd);
    return;
  }
  // pi/2 = 1.5707963267948966 + 6.123233995736766e-17 (the double nearest pi/2 and the
  // double nearest the rest)
  const double q = rint(theta * 0.63661977236758134);
  double r = fma(-q, 1.5707963267948966, theta);
  r = fma(-q, 6.123233995736766e-17, r);
  const float rh = (float)r;
  const ff sr = ff_make(rh, (float)(r - (double)rh));
  ff sn, cs;
  sincos_taylor_ff(sr, sn, cs);
  switch ((int)q & 3) {
    case 0:
      c = cs;
      s = sn;
      break;
    case 1:
      c = -sn;
      s = cs;
      break;
    case 2:
      c = -cs;
      s = -sn;
      break;
    default:
      c = sn;
      s = -cs;
      break;
  }
}

}  // namespace wp
