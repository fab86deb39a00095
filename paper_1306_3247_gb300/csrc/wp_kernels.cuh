// Device code of the split-operator step (Sec. 2.1 of arXiv:1306.3247), templated on
// the real type of the state (double: complex128 form; float: complex64 form).
//
// One kernel "pass" loads a tile of lines along one axis into shared memory, applies
// the operations selected by its flags (inverse FFT, potential phase, position sums,
// forward FFT, kinetic round trip, momentum sums) and writes the tile back. The FFT is
// a Stockham autosort transform with radix-8/4/2 butterflies held in registers; every
// stage reads and writes the tile in shared memory, so a pass touches HBM exactly once
// for reading and once for writing.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include <type_traits>

#include "wp_fft_f64.h"
#include "wp_ff.cuh"
#include "wp_phase_ff.cuh"
#include "wp_internal.h"

namespace wp {

// ------------------------------------------------------------------ complex helpers
template <class T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
  cx<T> r;
  r.re = a;
  r.im = b;
  return r;
}
template <class T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) {
  return mk(a.re + b.re, a.im + b.im);
}
template <class T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) {
  return mk(a.re - b.re, a.im - b.im);
}
template <class T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// a * conj(b)
template <class T>
__device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mk(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
// multiply by -i (forward transform) or +i (inverse transform)
template <class T, bool INV>
__device__ __forceinline__ cx<T> rot(cx<T> a) {
  return INV ? mk(-a.im, a.re) : mk(a.im, -a.re);
}

// Complex products in float-float: each real part is an error-free dot product of two
// terms (ff_dot2), cheaper than four ff products and two ff sums.
__device__ __forceinline__ cx<ff> cmul(cx<ff> a, cx<ff> b) {
  return mk(ff_dot2(a.re, b.re, a.im, b.im, -1.f), ff_dot2(a.re, b.im, a.im, b.re, 1.f));
}
__device__ __forceinline__ cx<ff> cmulc(cx<ff> a, cx<ff> b) {
  return mk(ff_dot2(a.re, b.re, a.im, b.im, 1.f), ff_dot2(a.im, b.re, a.re, b.im, -1.f));
}

// Real helpers of the line sums in the element type: zero, |v|^2, a b + c, warp exchange,
// conversion to FP64. Float-float uses error-free products and sums throughout.
template <class T>
__device__ __forceinline__ T tzero() {
  return T(0);
}
template <>
__device__ __forceinline__ ff tzero<ff>() {
  return ff_make(0.f, 0.f);
}
__device__ __forceinline__ float norm2(cx<float> v) { return fmaf(v.re, v.re, v.im * v.im); }
__device__ __forceinline__ double norm2(cx<double> v) { return fma(v.re, v.re, v.im * v.im); }
__device__ __forceinline__ ff norm2(cx<ff> v) { return ff_dot2(v.re, v.re, v.im, v.im, 1.f); }
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ ff madd(ff a, ff b, ff c) { return c + a * b; }
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ ff shfl_xor(ff v, int o) {
  return ff_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(ff v) { return (double)v; }

// ------------------------------------------------------------------ butterflies
// DFT of length R in registers, natural order in and out:
// X_k = sum_r x_r exp(-+ 2 pi i r k / R) (minus forward, plus inverse).
// Butterfly sums: the plain sums, and for float-float the unnormalised ones (cnorm
// renormalises the outputs of a butterfly).
template <class T>
__device__ __forceinline__ cx<T> cadd_b(cx<T> a, cx<T> b) {
  return cadd(a, b);
}
template <class T>
__device__ __forceinline__ cx<T> csub_b(cx<T> a, cx<T> b) {
  return csub(a, b);
}
template <class T>
__device__ __forceinline__ cx<T> cnorm(cx<T> a) {
  return a;
}
template <>
__device__ __forceinline__ cx<ff> cadd_b<ff>(cx<ff> a, cx<ff> b) {
  return mk(ff_add_raw(a.re, b.re), ff_add_raw(a.im, b.im));
}
template <>
__device__ __forceinline__ cx<ff> csub_b<ff>(cx<ff> a, cx<ff> b) {
  return mk(ff_add_raw(a.re, -b.re), ff_add_raw(a.im, -b.im));
}
template <>
__device__ __forceinline__ cx<ff> cnorm<ff>(cx<ff> a) {
  return mk(ff_norm(a.re), ff_norm(a.im));
}

__device__ __forceinline__ float radd(float a, float b) { return a + b; }
__device__ __forceinline__ double radd(double a, double b) { return a + b; }
__device__ __forceinline__ ff radd(ff a, ff b) { return ff_add_raw(a, b); }

template <class T, bool INV>
__device__ __forceinline__ void dft4_b(cx<T>& x0, cx<T>& x1, cx<T>& x2, cx<T>& x3) {
  cx<T> a0 = cadd_b(x0, x2), a1 = csub_b(x0, x2), a2 = cadd_b(x1, x3), a3 = rot<T, INV>(csub_b(x1, x3));
  x0 = cadd_b(a0, a2);
  x2 = csub_b(a0, a2);
  x1 = cadd_b(a1, a3);
  x3 = csub_b(a1, a3);
}

template <class T, bool INV>
__device__ __forceinline__ void dft4(cx<T>& x0, cx<T>& x1, cx<T>& x2, cx<T>& x3) {
  dft4_b<T, INV>(x0, x1, x2, x3);
  x0 = cnorm(x0);
  x1 = cnorm(x1);
  x2 = cnorm(x2);
  x3 = cnorm(x3);
}

template <class T, int R, bool INV>
struct Dft;

template <class T, bool INV>
struct Dft<T, 2, INV> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};

template <class T, bool INV>
struct Dft<T, 4, INV> {
  static __device__ __forceinline__ void run(cx<T>* v) { dft4<T, INV>(v[0], v[1], v[2], v[3]); }
};

// x / sqrt(2). The nearest float to 1/sqrt(2) is 1.7e-8 (relative) too small; applied to a
// quarter of the terms of every radix-8 stage that shrinks the norm by about 1e-8 per
// stage, coherently over the steps. In FP32 the product is therefore formed with a
// two-part constant hi + lo and the exact rounding error of hi*x (Dekker's two-product
// through an FMA), which leaves an unbiased, correctly rounded-or-nearly result. The
// rounded intrinsics keep the compiler from contracting the steps.
__device__ __forceinline__ double mul_rsqrt2(double x) { return 0.707106781186547524400844362104849039 * x; }
__device__ __forceinline__ ff mul_rsqrt2(ff x) {
  const float hi = 0.70710676908493042f, lo = 1.2101617e-8f;
  const float p = __fmul_rn(hi, x.hi);
  float e = fmaf(hi, x.hi, -p);
  e = fmaf(hi, x.lo, fmaf(lo, x.hi, e));
  return ff_fast_renorm(p, e);
}
__device__ __forceinline__ float mul_rsqrt2(float x) {
  const float hi = 0.70710676908493042f, lo = 1.2101617e-8f;
  const float p = __fmul_rn(hi, x);
  const float e = fmaf(hi, x, -p);
  return __fadd_rn(p, fmaf(lo, x, e));
}

template <class T, bool INV>
struct Dft<T, 8, INV> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    // radix-2 split into even and odd radix-4 transforms, combined with w8^k
    dft4_b<T, INV>(v[0], v[2], v[4], v[6]);
    dft4_b<T, INV>(v[1], v[3], v[5], v[7]);
    cx<T> o1 = v[3], o2 = v[5], o3 = v[7];
    cx<T> t1 = INV ? mk(mul_rsqrt2(radd(o1.re, -o1.im)), mul_rsqrt2(radd(o1.re, o1.im)))
                   : mk(mul_rsqrt2(radd(o1.re, o1.im)), mul_rsqrt2(radd(o1.im, -o1.re)));
    cx<T> t2 = rot<T, INV>(o2);
    cx<T> t3 = INV ? mk(-mul_rsqrt2(radd(o3.re, o3.im)), mul_rsqrt2(radd(o3.re, -o3.im)))
                   : mk(mul_rsqrt2(radd(o3.im, -o3.re)), -mul_rsqrt2(radd(o3.re, o3.im)));
    cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cnorm(cadd_b(e0, o0));
    v[4] = cnorm(csub_b(e0, o0));
    v[1] = cnorm(cadd_b(e1, t1));
    v[5] = cnorm(csub_b(e1, t1));
    v[2] = cnorm(cadd_b(e2, t2));
    v[6] = cnorm(csub_b(e2, t2));
    v[3] = cnorm(cadd_b(e3, t3));
    v[7] = cnorm(csub_b(e3, t3));
  }
};

template <int R>
struct Log2R;
template <>
struct Log2R<2> {
  static constexpr int v = 1;
};
template <>
struct Log2R<4> {
  static constexpr int v = 2;
};
template <>
struct Log2R<8> {
  static constexpr int v = 3;
};

// Products with a factor stored as high + low parts (FP32 tables). The rounded table
// entries have |w_h| != 1 by up to 6e-8; the same entries act on the same part of the
// data every step, so a fixed modulus error accumulates into a steady norm drift. The low
// part is folded into the FMA chain before the final rounding, so each result is the
// rounded value of v (w_h + w_l) and the remaining rounding error is unbiased. (Adding
// v w_l to an already rounded v w_h would lose it: it is below half an ulp.)
__device__ __forceinline__ cx<float> cmul2(cx<float> v, cx<float> h, cx<float> l) {
  const float cr = v.re * l.re - v.im * l.im;
  const float ci = v.re * l.im + v.im * l.re;
  return mk(fmaf(v.re, h.re, fmaf(-v.im, h.im, cr)), fmaf(v.re, h.im, fmaf(v.im, h.re, ci)));
}
// v * conj(h + l)
__device__ __forceinline__ cx<float> cmulc2(cx<float> v, cx<float> h, cx<float> l) {
  const float cr = v.re * l.re + v.im * l.im;
  const float ci = v.im * l.re - v.re * l.im;
  return mk(fmaf(v.re, h.re, fmaf(v.im, h.im, cr)), fmaf(v.im, h.re, fmaf(-v.re, h.im, ci)));
}

// Twiddle multiplication v * w (forward) or v * conj(w) (inverse). FP64 uses the
// table entry directly.
template <bool INV>
__device__ __forceinline__ cx<double> twiddle(cx<double> v, const cx<double>* __restrict__ W,
                                              const cx<double>* __restrict__, int k) {
  const cx<double> w = W[k];
  return INV ? cmulc(v, w) : cmul(v, w);
}
template <bool INV>
__device__ __forceinline__ cx<ff> twiddle(cx<ff> v, const cx<ff>* __restrict__ W, const cx<ff>* __restrict__,
                                          int k) {
  const cx<ff> w = W[k];
  return INV ? cmulc(v, w) : cmul(v, w);
}
template <bool INV>
__device__ __forceinline__ cx<float> twiddle(cx<float> v, const cx<float>* __restrict__ W,
                                             const cx<float>* __restrict__ Wl, int k) {
  return INV ? cmulc2(v, W[k], Wl[k]) : cmul2(v, W[k], Wl[k]);
}

// ------------------------------------------------------------------ tile FFT
// Shared-memory tile: element i of line l at s[i * LS + l], C = 2^logC lines of
// n = 2^logn elements. Thread mapping puts lines fastest, so a warp touches
// consecutive addresses in every stage.
//
// One Stockham stage of radix R with current span Ns (Ns = product of the radices of
// the previous stages): butterfly j reads x[j + r n/R], multiplies by the twiddle
// w_{Ns R}^{r (j mod Ns)}, transforms, and writes to (j div Ns) Ns R + (j mod Ns) + r Ns.
// After the last stage the line holds its DFT in natural order.
template <class T, int R, int E, bool INV>
__device__ __forceinline__ void fft_stage(cx<T>* s, int logn, int logC, int LS, int logNs,
                                          const cx<T>* __restrict__ W, const cx<T>* __restrict__ Wl, int tid,
                                          int nthr) {
  constexpr int B = E / R;
  constexpr int LR = Log2R<R>::v;
  const int C = 1 << logC;
  const int nR = 1 << (logn - LR);
  const int total = C << (logn - LR);
  const int Nsm = (1 << logNs) - 1;
  const int twlog = logn - logNs - LR;
  cx<T> v[B][R];
#pragma unroll
  for (int b = 0; b < B; b++) {
    const int bi = tid + b * nthr;
    if (bi < total) {
      const int l = bi & (C - 1), j = bi >> logC;
#pragma unroll
      for (int r = 0; r < R; r++) v[b][r] = s[(j + r * nR) * LS + l];
      if (logNs > 0) {
        const int jm = j & Nsm;
#pragma unroll
        for (int r = 1; r < R; r++) v[b][r] = twiddle<INV>(v[b][r], W, Wl, (r * jm) << twlog);
      }
      Dft<T, R, INV>::run(v[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < B; b++) {
    const int bi = tid + b * nthr;
    if (bi < total) {
      const int l = bi & (C - 1), j = bi >> logC;
      const int jm = j & Nsm;
      const int d0 = ((j >> logNs) << (logNs + LR)) + jm;
#pragma unroll
      for (int r = 0; r < R; r++) s[(d0 + (r << logNs)) * LS + l] = v[b][r];
    }
  }
  __syncthreads();
}

// Whole-line transform of every line of the tile (unnormalised).
// maxr: log2 of the largest butterfly (3: radix 8 while at least 5 or exactly 3 factors of
// two remain, then 4, then 2; 2: radix 4 then 2).
template <class T, int E, bool INV>
__device__ void fft_tile(cx<T>* s, int logn, int logC, int LS, const cx<T>* __restrict__ W,
                         const cx<T>* __restrict__ Wl, int tid, int nthr, int maxr = 3) {
  int logNs = 0;
  while (logNs < logn) {
    const int rem = logn - logNs;
    if (E >= 8 && maxr >= 3 && (rem >= 5 || rem == 3)) {
      fft_stage<T, 8, E, INV>(s, logn, logC, LS, logNs, W, Wl, tid, nthr);
      logNs += 3;
    } else if (E >= 4 && rem >= 2) {
      fft_stage<T, 4, E, INV>(s, logn, logC, LS, logNs, W, Wl, tid, nthr);
      logNs += 2;
    } else {
      fft_stage<T, 2, E, INV>(s, logn, logC, LS, logNs, W, Wl, tid, nthr);
      logNs += 1;
    }
  }
}

// ------------------------------------------------------------------ fixed-size tile FFT
// The same Stockham stages with n, C and the row stride known at compile time. Stage
// twiddles come from a per-stage table: for the stage with span Ns and radix R, entry
// jm (R-1) + r - 1 holds w_n^{r jm n/(Ns R)}, so one butterfly reads its R-1 twiddles as
// consecutive 16-byte records. The stage plan is wp_stage_radix_log, shared with the host
// code that builds the table.
template <bool INV>
__device__ __forceinline__ cx<double> tw_apply(cx<double> v, const TwE<double>& e) {
  return INV ? cmulc(v, e.w) : cmul(v, e.w);
}
template <bool INV>
__device__ __forceinline__ cx<ff> tw_apply(cx<ff> v, const TwE<ff>& e) {
  return INV ? cmulc(v, e.w) : cmul(v, e.w);
}
template <bool INV>
__device__ __forceinline__ cx<float> tw_apply(cx<float> v, const TwE<float>& e) {
  return INV ? cmulc2(v, e.h, e.l) : cmul2(v, e.h, e.l);
}

template <class T, int LOGN, int LOGC, int LS, int LOGNS, bool INV, int EPT = 8>
__device__ __forceinline__ void stage_fixed(cx<T>* s, const TwE<T>* __restrict__ tw, int tid) {
  constexpr int LR = wp_stage_radix_log(LOGN, LOGNS);
  constexpr int R = 1 << LR;
  constexpr int C = 1 << LOGC;
  constexpr int NR = 1 << (LOGN - LR);
  constexpr int NT = (C << LOGN) / EPT;  // threads: EPT elements each
  constexpr int B = EPT / R;
  constexpr int NS = 1 << LOGNS;
  cx<T> v[B][R];
#pragma unroll
  for (int b = 0; b < B; b++) {
    const int bi = tid + b * NT;
    const int l = bi & (C - 1), j = bi >> LOGC;
#pragma unroll
    for (int r = 0; r < R; r++) v[b][r] = s[(j + r * NR) * LS + l];
    if (LOGNS > 0) {
      const TwE<T>* e = tw + (j & (NS - 1)) * (R - 1);
#pragma unroll
      for (int r = 1; r < R; r++) v[b][r] = tw_apply<INV>(v[b][r], e[r - 1]);
    }
    Dft<T, R, INV>::run(v[b]);
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < B; b++) {
    const int bi = tid + b * NT;
    const int l = bi & (C - 1), j = bi >> LOGC;
    const int d0 = ((j >> LOGNS) << (LOGNS + LR)) + (j & (NS - 1));
#pragma unroll
    for (int r = 0; r < R; r++) s[(d0 + (r << LOGNS)) * LS + l] = v[b][r];
  }
  __syncthreads();
}

// The FP64 stages in fused multiply-add form (wp_fft_f64.h): the same loads, stores and
// stage plan; the butterflies read their twiddle records from the direction's table.
template <int LOGN, int LOGC, int LS, int LOGNS, bool INV, int EPT = 8>
__device__ __forceinline__ void stage_fixed_f64(cx<double>* s, const unsigned char* __restrict__ tab, int tid) {
  constexpr int LR = wp_stage_radix_log(LOGN, LOGNS);
  constexpr int R = 1 << LR;
  constexpr int C = 1 << LOGC;
  constexpr int NR = 1 << (LOGN - LR);
  constexpr int NT = (C << LOGN) / EPT;  // threads: EPT elements each
  constexpr int B = EPT / R;
  constexpr int NS = 1 << LOGNS;
  constexpr int OFF = (INV ? wp_fma_dir_bytes(LOGN) : 0) + wp_fma_stage_offset(LOGN, LOGNS);
  constexpr int RB = wp_fma_rec_bytes(LR);
  cx<double> v[B][R];
#pragma unroll
  for (int b = 0; b < B; b++) {
    const int bi = tid + b * NT;
    const int l = bi & (C - 1), j = bi >> LOGC;
#pragma unroll
    for (int r = 0; r < R; r++) v[b][r] = s[(j + r * NR) * LS + l];
    if constexpr (LOGNS == 0) {
      if constexpr (R == 8)
        fma_dft8_first<INV>(v[b]);
      else
        Dft<double, R, INV>::run(v[b]);
    } else {
      const unsigned char* rec = tab + OFF + (j & (NS - 1)) * RB;
      if constexpr (R == 8)
        fma_dft8<INV>(v[b], *reinterpret_cast<const Fma8*>(rec));
      else if constexpr (R == 4)
        fma_dft4<INV>(v[b], *reinterpret_cast<const Fma4*>(rec));
      else
        fma_dft2<INV>(v[b], *reinterpret_cast<const Fma2*>(rec));
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < B; b++) {
    const int bi = tid + b * NT;
    const int l = bi & (C - 1), j = bi >> LOGC;
    const int d0 = ((j >> LOGNS) << (LOGNS + LR)) + (j & (NS - 1));
#pragma unroll
    for (int r = 0; r < R; r++) s[(d0 + (r << LOGNS)) * LS + l] = v[b][r];
  }
  __syncthreads();
}

// tw: the per-stage records of the axis, 2^LOGN 16-byte entries; for FP64 the fused
// multiply-add records of both directions follow them. FMA: use those (FP64 only; the
// resident 1-D lines keep the product form, whose register needs fit their blocks).
template <class T, int LOGN, int LOGC, int LS, bool INV, int LOGNS, int EPT = 8,
          bool FMA = std::is_same<T, double>::value>
__device__ __forceinline__ void fft_fixed(cx<T>* s, const TwE<T>* __restrict__ tw, int tid) {
  if constexpr (LOGNS < LOGN) {
    if constexpr (FMA)
      stage_fixed_f64<LOGN, LOGC, LS, LOGNS, INV, EPT>(s, reinterpret_cast<const unsigned char*>(tw + (1 << LOGN)),
                                                       tid);
    else
      stage_fixed<T, LOGN, LOGC, LS, LOGNS, INV, EPT>(s, tw + wp_stage_tw_offset(LOGN, LOGNS), tid);
    fft_fixed<T, LOGN, LOGC, LS, INV, LOGNS + wp_stage_radix_log(LOGN, LOGNS), EPT, FMA>(s, tw, tid);
  }
}

// ------------------------------------------------------------------ reductions
// Fixed-order block sum of NQ doubles; thread 0 of the block receives the totals in
// out[0..NQ). Every thread must call it. Deterministic for a fixed launch shape.
__device__ __forceinline__ void block_sum(double (&acc)[NQ], double* out, double (*red)[NQ]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; q++) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double v = 0.0;
    for (int w = 0; w < nwarps; w++) v += red[w][threadIdx.x];
    out[threadIdx.x] = v;
  }
  __syncthreads();
}

// Observable record from the position sums qp and momentum sums qm (Tab. 3):
// 0 t, 1 norm, 2-4 <x>, 5-7 <p>, 8-10 <x^2>, 11 E, 12 E_K, 13 E_V, 14 autocorrelation, 15 step.
__device__ inline void finish_obs(const double* qp, const double* qm, const Geom& g, int64_t ntotal,
                                  int autocorr, double t, int64_t step, double* rec) {
  const double dv = g.dv;
  const double dvk = dv / (double)ntotal;
  rec[0] = t;
  rec[1] = sqrt(qp[Q_RHO] * dv);
  for (int d = 0; d < 3; d++) {
    rec[2 + d] = qp[Q_X + d] * dv;
    rec[5 + d] = g.hbar * qm[Q_K + d] * dvk;
    rec[8 + d] = qp[Q_XX + d] * dv;
  }
  rec[12] = g.hbar * g.hbar / (2.0 * g.mass) * qm[Q_K2] * dvk;
  rec[13] = qp[Q_V] * dv;
  rec[11] = rec[12] + rec[13];
  rec[14] = autocorr ? (qp[Q_AC_RE] * qp[Q_AC_RE] + qp[Q_AC_IM] * qp[Q_AC_IM]) * dv * dv : 0.0;
  rec[15] = (double)step;
}

// ------------------------------------------------------------------ potential terms
// f(t) = A0 + A env(t) sin(omega t + phi)
__device__ inline double term_coef(const wp_pot_term& tm, double t) {
  double env = 1.0;
  if (tm.env == WP_ENV_GAUSS) {
    const double u = (t - tm.t0) / tm.tau;
    env = exp(-u * u);
  } else if (tm.env == WP_ENV_SIN2) {
    if (t >= tm.t0 && t <= tm.t0 + tm.tau) {
      const double sv = sin(3.14159265358979323846 * t / tm.tau);
      env = sv * sv;
    } else {
      env = 0.0;
    }
  }
  return tm.A0 + tm.A * env * sin(tm.omega * t + tm.phi);
}

// Additive (non-Gaussian) shape restricted to axis d: the potential is the sum of
// these per-axis parts plus the Gaussian products.
__device__ inline double term_axis_part(const wp_pot_term& tm, int d, double x, double t) {
  const double u = x - (tm.c0[d] + tm.v[d] * t);
  switch (tm.shape) {
    case WP_SHAPE_CONST:
      return d == 0 ? 1.0 : 0.0;
    case WP_SHAPE_QUAD:
      return 0.5 * tm.a[d] * u * u;
    case WP_SHAPE_LINEAR:
      return tm.a[d] * u;
    case WP_SHAPE_MORSE:
      if ((int)tm.a[2] == d) {
        const double e = 1.0 - exp(-tm.a[1] * u);
        return tm.a[0] * e * e;
      }
      return 0.0;
    default:
      return 0.0;
  }
}

__device__ inline double gauss_axis_factor(const wp_pot_term& tm, int d, double x, double t) {
  if (!(tm.a[d] > 0.0)) return 1.0;
  const double u = (x - (tm.c0[d] + tm.v[d] * t)) / tm.a[d];
  return exp(-u * u);
}

// Index of element i along axis `axis`, outer line index o (axes before) and inner
// index c (axes after) -> grid indices gi[0..2].
__device__ __forceinline__ void grid_index(const Geom& g, int axis, int64_t o, int64_t c, int i, int gi[3]) {
  gi[0] = gi[1] = gi[2] = 0;
  gi[axis] = i;
  for (int d = g.ndim - 1; d > axis; d--) {
    gi[d] = (int)(c & ((1 << g.ln[d]) - 1));
    c >>= g.ln[d];
  }
  for (int d = axis - 1; d >= 0; d--) {
    gi[d] = (int)(o & ((1 << g.ln[d]) - 1));
    o >>= g.ln[d];
  }
}

__device__ __forceinline__ double wavenumber(const Geom& g, int d, int j) {
  const int n = 1 << g.ln[d];
  const int js = j < (n >> 1) ? j : j - n;
  return g.kscale[d] * (double)js;
}

// ------------------------------------------------------------------ factor application
// A phase factor is the product of the pass-axis table entry a (element dependent) and
// the per-line product L of the other axes' entries; both are stored as high + low parts,
// L formed in FP64. In FP32 the product a L is first formed as high + low parts
// (error-free products and sums), then applied to v with a single rounding (cmul2).
// Two successive roundings (v a, then (v a) L) were measured to leave a norm drift near
// 1e-8 per step on stationary packets; one rounding of the exact factor leaves 1e-10.
// In FP64 the plain product is accurate enough.
__device__ __forceinline__ cx<double> apply_factor(cx<double> v, cx<double> ah, cx<double>, cx<double> Lh,
                                                   cx<double>) {
  return cmul(v, cmul(ah, Lh));
}

__device__ __forceinline__ cx<ff> apply_factor(cx<ff> v, cx<ff> ah, cx<ff>, cx<ff> Lh, cx<ff>) {
  return cmul(v, cmul(ah, Lh));
}

// a*b - c*d as s + err, err exact to O(eps^2) (Dekker products through FMA, Knuth sum).
__device__ __forceinline__ void diff_of_products(float a, float b, float c, float d, float& s, float& err) {
  const float p = __fmul_rn(a, b), q = __fmul_rn(c, d);
  const float ep = fmaf(a, b, -p), eq = fmaf(c, d, -q);
  s = __fsub_rn(p, q);
  const float bb = __fsub_rn(s, p);
  const float es = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(-q, bb));
  err = __fadd_rn(__fsub_rn(ep, eq), es);
}

__device__ __forceinline__ cx<float> apply_factor(cx<float> v, cx<float> ah, cx<float> al, cx<float> Lh,
                                                  cx<float> Ll) {
  cx<float> fh, fl;
  float e;
  diff_of_products(ah.re, Lh.re, ah.im, Lh.im, fh.re, e);
  fl.re = e + (fmaf(ah.re, Ll.re, al.re * Lh.re) - fmaf(ah.im, Ll.im, al.im * Lh.im));
  diff_of_products(ah.re, Lh.im, -ah.im, Lh.re, fh.im, e);
  fl.im = e + (fmaf(ah.re, Ll.im, al.re * Lh.im) + fmaf(ah.im, Ll.re, al.im * Lh.re));
  return cmul2(v, fh, fl);
}

// exp(-i theta) applied to v. In FP32 the factor is written as 1 + (c - 1) - i s with
// c - 1 = -2 sin^2(theta/2), whose modulus is 1 up to O(eps theta^2).
// FP64: Taylor series of sin and cos, to theta^5 / theta^6 for |theta| < 2^-8 (below
// 1e-18 relative; the usual barrier phase per step) and to theta^9 / theta^10 for
// |theta| < 1/16 (below 1e-20); larger arguments use the library sincos.
__device__ __forceinline__ cx<double> apply_gauss_phase(cx<double> v, double th) {
  // a localised term leaves most points with |theta| < 2^-60, where the factor is 1 to
  // below 1e-18 relative: those points are left as they are
  if (fabs(th) < 0x1p-60) return v;
  double sn, cs;
  if (fabs(th) < 0.00390625) {
    const double z = th * th;
    sn = th * (1.0 + z * (-1.0 / 6 + z * (1.0 / 120)));
    cs = 1.0 + z * (-0.5 + z * (1.0 / 24 + z * (-1.0 / 720)));
  } else if (fabs(th) < 0.0625) {
    const double z = th * th;
    sn = th * (1.0 + z * (-1.0 / 6 + z * (1.0 / 120 + z * (-1.0 / 5040 + z * (1.0 / 362880)))));
    cs = 1.0 + z * (-0.5 + z * (1.0 / 24 + z * (-1.0 / 720 + z * (1.0 / 40320 + z * (-1.0 / 3628800)))));
  } else {
    sincos(th, &sn, &cs);
  }
  return cmul(v, mk(cs, -sn));
}
// Float-float: the same two Taylor tiers in float-float arithmetic, the FP64 sincos
// otherwise.
__device__ __forceinline__ cx<ff> apply_gauss_phase(cx<ff> v, ff th) {
  if (fabsf(th.hi) < 0x1p-56f) return v;  // the factor is 1 to below the pair's precision
  ff sn, cs;
  if (fabsf(th.hi) < 0.00390625f) {
    // |theta| < 2^-8: terms to theta^5 / theta^6 (below 1e-18 relative)
    const ff z = th * th;
    sn = th * (ff(1.0) + z * (ff(-1.0 / 6) + z * ff(1.0 / 120)));
    cs = ff(1.0) + z * (ff(-0.5) + z * (ff(1.0 / 24) + z * ff(-1.0 / 720)));
  } else if (fabsf(th.hi) < 0.0625f) {
    const ff z = th * th;
    sn = th * (ff(1.0) + z * (ff(-1.0 / 6) + z * (ff(1.0 / 120) + z * (ff(-1.0 / 5040) + z * ff(1.0 / 362880)))));
    cs = ff(1.0) + z * (ff(-0.5) + z * (ff(1.0 / 24) + z * (ff(-1.0 / 720) + z * (ff(1.0 / 40320) +
                                                                                      z * ff(-1.0 / 3628800)))));
  } else {
    double s, c;
    sincos((double)th, &s, &c);
    sn = ff(s);
    cs = ff(c);
  }
  return cmul(v, mk(cs, -sn));
}
__device__ __forceinline__ cx<float> apply_gauss_phase(cx<float> v, float th) {
  float sh, ch;
  const float h = 0.5f * th;
  if (fabsf(h) < 0x1p-26f) return v;  // v g is below half an ulp of v
  if (fabsf(h) < 0.03125f) {
    // Taylor series of sin and cos at h (terms to h^7 / h^6 leave < 1e-15 relative)
    const float z = h * h;
    sh = h * (1.0f + z * (-1.0f / 6 + z * (1.0f / 120 - z * (1.0f / 5040))));
    ch = 1.0f + z * (-0.5f + z * (1.0f / 24 - z * (1.0f / 720)));
  } else {
    sincosf(h, &sh, &ch);
  }
  const cx<float> g = mk(-2.0f * sh * sh, -2.0f * sh * ch);
  return cadd(v, cmul(v, g));
}

// A Gaussian term whose line coefficient g is below the level where apply_gauss_phase
// leaves a point as it is (FP64 |theta| < 2^-60, float-float 2^-56, FP32 2^-25) gives every
// point of the line such a phase (theta = g x axis factor, and the axis factors are at most
// 1): the whole line can skip that term, with the same result. For a localised barrier that
// is almost every line.
__device__ __forceinline__ bool gauss_line_active(double g) { return fabs(g) >= 0x1p-60; }
__device__ __forceinline__ bool gauss_line_active(float g) { return fabsf(g) >= 0x1p-25f; }
__device__ __forceinline__ bool gauss_line_active(ff g) { return fabsf(g.hi) >= 0x1p-57f; }

// Record forms of apply_factor (fixed-size kernels).
__device__ __forceinline__ cx<double> apply_factor_rec(cx<double> v, const TwE<double>& a, const TwE<double>& L) {
  return cmul(v, cmul(a.w, L.w));
}
__device__ __forceinline__ cx<ff> apply_factor_rec(cx<ff> v, const TwE<ff>& a, const TwE<ff>& L) {
  return cmul(v, cmul(a.w, L.w));
}
__device__ __forceinline__ cx<float> apply_factor_rec(cx<float> v, const TwE<float>& a, const TwE<float>& L) {
  return apply_factor(v, a.h, a.l, L.h, L.l);
}

// Per-line products of the non-pass axes' factors (FP64, split into high and low parts),
// and of the Gaussian-term factors times their coefficient.
template <class T>
__device__ void line_factors(const PassParams<T>& p, const cx<T>* const* H, const cx<T>* const* Lo, bool gauss,
                             bool contig, int64_t o0, int64_t cb, int C, cx<T>* sLh, cx<T>* sLl,
                             T (*sGl)[64]) {
  for (int l = threadIdx.x; l < C; l += blockDim.x) {
    int gi[3];
    if (contig)
      grid_index(p.g, p.axis, o0 + l, 0, 0, gi);
    else
      grid_index(p.g, p.axis, o0, cb + l, 0, gi);
    double r = 1.0, m = 0.0;
    for (int d = 0; d < p.g.ndim; d++) {
      if (d == p.axis) continue;
      const cx<T> hh = H[d][gi[d]], ll = Lo[d][gi[d]];
      const double fr = (double)hh.re + (double)ll.re, fi = (double)hh.im + (double)ll.im;
      const double nr = r * fr - m * fi, ni = r * fi + m * fr;
      r = nr;
      m = ni;
    }
    const T hr = (T)r, hm = (T)m;
    sLh[l] = mk(hr, hm);
    sLl[l] = mk((T)(r - (double)hr), (T)(m - (double)hm));
    if (gauss) {
      for (int gg = 0; gg < p.ngauss; gg++) {
        double prod = p.ctrl->gphase[gg];
        for (int d = 0; d < p.g.ndim; d++)
          if (d != p.axis) prod *= p.Gd[gg][d][gi[d]];
        sGl[gg][l] = (T)prod;
      }
    }
  }
}

// ------------------------------------------------------------------ pass kernel
// Shape of a pass: tile lines C = 2^logC, line length n = 2^logn, shared-memory row
// stride LS, contiguous or strided axis, block size. DynShape holds them at run time;
// FixShape makes them compile-time constants so that every index folds and the stage
// sequence unrolls (used for n = 64..1024, the common grid sizes).
struct DynShape {
  static constexpr bool fixed = false;
  int logn, logC, LS, nthr;
  bool contig;
  template <class T>
  __device__ explicit DynShape(const PassParams<T>& p)
      : logn(p.logn), logC(p.logC), LS(p.LS), nthr(p.nthreads), contig(p.log_inner == 0) {}
};

template <int LOGN, bool CONTIG>
struct FixShape {
  static constexpr bool fixed = true;                      // reads per-line records
  static constexpr int logn = LOGN;
  static constexpr int logC = 11 - LOGN;                   // 2048-element tiles
  static constexpr int LS = 1 << logC;
  static constexpr int nthr = 256;                         // 8 elements per thread
  static constexpr bool contig = CONTIG;
};

// Transforms of the tile: the run-time Stockham loop, or the unrolled fixed-size one with
// per-stage twiddle tables.
template <class T, int E, bool INV>
__device__ __forceinline__ void tile_fft(cx<T>* s, const PassParams<T>& p, const DynShape& sh, int tid) {
  fft_tile<T, E, INV>(s, sh.logn, sh.logC, sh.LS, p.W, p.W_lo, tid, sh.nthr, p.max_radix_log);
}
template <class T, int E, bool INV, int LOGN, bool CONTIG>
__device__ __forceinline__ void tile_fft(cx<T>* s, const PassParams<T>& p, const FixShape<LOGN, CONTIG>&, int tid) {
  using SH = FixShape<LOGN, CONTIG>;
  fft_fixed<T, SH::logn, SH::logC, SH::LS, INV, 0>(s, reinterpret_cast<const TwE<T>*>(p.Wst), tid);
}

// Global line coordinates of tile `tile`: contiguous axis -> lines o0 .. o0 + C - 1;
// strided axis -> outer index o0, columns cb .. cb + C - 1.
template <class T, class SH>
__device__ __forceinline__ void tile_origin(const PassParams<T>& p, const SH& sh, int64_t tile, int64_t& o0,
                                            int64_t& cb) {
  if (sh.contig) {
    o0 = tile << sh.logC;
    cb = 0;
  } else {
    const int tpo = p.log_inner - sh.logC;
    o0 = tile >> tpo;
    cb = (tile & ((int64_t(1) << tpo) - 1)) << sh.logC;
  }
}

// Element (i, l) of the tile <-> global index. Loads and stores run with the lines
// fastest: a warp touches 32 / C consecutive points of each of C lines (contiguous axis:
// C full sectors; strided axis: one row segment of C adjacent columns) and consecutive
// shared-memory words.
template <class T, class SH>
__device__ __forceinline__ int64_t tile_gidx(const PassParams<T>& p, const SH& sh, int64_t o0, int64_t cb, int i,
                                             int l) {
  return sh.contig ? ((o0 + l) << sh.logn) + i : (((o0 << sh.logn) + i) << p.log_inner) + cb + l;
}

// Fixed-shape tiles: 256 threads, 2048 elements. Thread t always serves line
// l = t mod C and the points i = t / C + k 256 / C (k = 0..7), so its global addresses are a
// base pointer plus a constant stride: no per-element 64-bit index arithmetic.
template <class T, class SH>
__device__ __forceinline__ void fixed_walk(const PassParams<T>& p, int64_t o0, int64_t cb, int& l, int& i0,
                                           int64_t& base, int64_t& estride) {
  l = threadIdx.x & ((1 << SH::logC) - 1);
  i0 = threadIdx.x >> SH::logC;
  if (SH::contig) {
    base = ((o0 + l) << SH::logn) + i0;
    estride = 1;
  } else {
    estride = int64_t(1) << p.log_inner;
    base = (((o0 << SH::logn) + i0) << p.log_inner) + cb + l;
  }
}

template <class T, class SH>
__device__ __forceinline__ void fixed_load(const PassParams<T>& p, cx<T>* s, int64_t tile) {
  constexpr int ISTEP = 256 >> SH::logC;
  int64_t o0, cb;
  tile_origin(p, SH(), tile, o0, cb);
  int l, i0;
  int64_t base, es;
  fixed_walk<T, SH>(p, o0, cb, l, i0, base, es);
  const cx<T>* src = p.in + base;
  const int64_t step = es * ISTEP;
  cx<T> v[8];
#pragma unroll
  for (int k = 0; k < 8; k++) v[k] = src[k * step];
#pragma unroll
  for (int k = 0; k < 8; k++) s[(i0 + k * ISTEP) * SH::LS + l] = v[k];
}

// One line's part of the 16 observable sums in FP64 (Tab. 3 quantities), from its sums
// lt[0..7] over the pass axis (position pass: |psi|^2 times 1, x, x^2, the additive
// potential, the Gaussian axis factors, and <psi0|psi>; momentum pass: |psi_hat|^2 times
// 1, k, k^2) and its grid index gi on the other axes: the pass-axis moments come from the
// line sums, the other axes' coordinates, wavenumbers, potential parts and Gaussian
// factors are constant along the line (the potential is a sum of per-axis parts and
// products of per-axis Gaussian factors).
template <class T>
__device__ __forceinline__ void obs_line_row(const PassParams<T>& p, const double (&lt)[8], const int (&gi)[3],
                                             double* c) {
  const int ax = p.axis;
  for (int k = 0; k < NQ; k++) c[k] = 0.0;
  if (p.flags & F_OBS_POS) {
    c[Q_RHO] = lt[0];
    const double xs = p.g.oscale_x[ax];  // the tables hold x / xs
    c[Q_X + ax] = lt[1] * xs;
    c[Q_XX + ax] = lt[2] * (xs * xs);
    double A = 0.0;
    for (int d = 0; d < p.g.ndim; d++) {
      if (d == ax) continue;
      const double x = p.g.xmin[d] + (double)gi[d] * p.g.dx[d];
      c[Q_X + d] = x * lt[0];
      c[Q_XX + d] = x * x * lt[0];
      A += p.A[d][gi[d]];
    }
    double v = lt[3] + A * lt[0];
    for (int gg = 0; gg < p.ngauss; gg++) {
      double prod = p.ctrl->gcoef[gg];
      for (int d = 0; d < p.g.ndim; d++)
        if (d != ax) prod *= p.Gd[gg][d][gi[d]];
      v += prod * lt[4 + gg];
    }
    c[Q_V] = v;
    c[Q_AC_RE] = lt[6];
    c[Q_AC_IM] = lt[7];
  } else {
    c[Q_RHOK] = lt[0];
    const double ks = p.g.oscale_k[ax];  // the tables hold k / ks
    c[Q_K + ax] = lt[1] * ks;
    double k2 = 0.0;
    for (int d = 0; d < p.g.ndim; d++) {
      if (d == ax) continue;
      const double k = wavenumber(p.g, d, gi[d]);
      c[Q_K + d] = k * lt[0];
      k2 += k * k;
    }
    c[Q_K2] = lt[2] * (ks * ks) + k2 * lt[0];
  }
}

// Block partials of the observable sums in a fixed-size kernel. Thread t holds the sums
// of line l = t mod C over its 8 points (q[0..7], in T). The lanes of a line are combined
// by xor shuffles, the 8 warps through the tile buffer, in a fixed order; each line adds
// its row (obs_line_row). Partials of block b go to partials[b].
template <class T, class SH>
__device__ __forceinline__ void fixed_obs_reduce(const PassParams<T>& p, T (&q)[8], int64_t o0, int64_t cb,
                                                 T* scratch, double (*red)[NQ]) {
  constexpr int C = 1 << SH::logC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int o = C; o < 32; o <<= 1)
#pragma unroll
    for (int j = 0; j < 8; j++) q[j] = q[j] + shfl_xor(q[j], o);
  if (lane < C)
#pragma unroll
    for (int j = 0; j < 8; j++) scratch[(warp * C + lane) * 8 + j] = q[j];
  __syncthreads();
  if (tid < 8 * C) {
    const int l = tid >> 3, j = tid & 7;
    T sum = scratch[l * 8 + j];
#pragma unroll
    for (int w = 1; w < 8; w++) sum = sum + scratch[(w * C + l) * 8 + j];
    red[l][j] = to_f64(sum);
  }
  __syncthreads();
  double lt[8];
  if (tid < C)
#pragma unroll
    for (int j = 0; j < 8; j++) lt[j] = red[tid][j];
  __syncthreads();
  if (tid < C) {
    int gi[3];
    if (SH::contig)
      grid_index(p.g, p.axis, o0 + tid, 0, 0, gi);
    else
      grid_index(p.g, p.axis, o0, cb + tid, 0, gi);
    obs_line_row(p, lt, gi, red[tid]);
  }
  __syncthreads();
  if (tid < NQ) {
    double sum = 0.0;
    for (int l = 0; l < C; l++) sum += red[l][tid];
    p.partials[blockIdx.x * (int64_t)NQ + tid] = sum;
  }
}

// Everything a pass does once its tile is in shared memory: the transforms and factors
// selected by the flags, the store, the partial sums. Ends with a block barrier.
template <class T, int E, bool OBS, class SH, bool GRID = false>
__device__ __forceinline__ void pass_compute(const PassParams<T>& p, const SH& sh, cx<T>* s, int64_t tile) {
  __shared__ double red[32][NQ];
  __shared__ double tot[NQ];
  __shared__ cx<T> sLh[64], sLl[64];
  __shared__ T sGl[WP_MAX_GAUSS][64];
  __shared__ LineRec<T> sRec[64];
  const int tid = threadIdx.x;
  const int nthr = sh.nthr;
  const int logn = sh.logn, logC = sh.logC, LS = sh.LS;
  const int C = 1 << logC;
  const bool contig = sh.contig;
  int64_t o0, cb;
  tile_origin(p, sh, tile, o0, cb);
  const int ntot = C << logn;

  const uint32_t f = p.flags;
  if (f & F_IFFT) tile_fft<T, E, true>(s, p, sh, tid);

  double acc[NQ];
#pragma unroll
  for (int k = 0; k < NQ; k++) acc[k] = 0.0;
  T q[8];  // fixed-size kernels: the thread's line sums
#pragma unroll
  for (int k = 0; k < 8; k++) q[k] = tzero<T>();

  if (f & (F_PHASE | (OBS ? F_OBS_POS : 0u))) {
    if (f & F_PHASE) {
      if constexpr (SH::fixed) {
        for (int l = tid; l < C; l += nthr) sRec[l] = p.lines_phase[contig ? o0 + l : cb + l];
      } else {
        line_factors<T>(p, p.P, p.P_lo, true, contig, o0, cb, C, sLh, sLl, sGl);
      }
      __syncthreads();
    }
    const cx<T>* Pa = p.P[p.axis];
    const cx<T>* Pal = p.P_lo[p.axis];
    if constexpr (SH::fixed) {
      // thread-fixed line record, points i0 + k 256/C; with OBS also the thread's line
      // sums of |psi|^2 times 1, x, x^2, A(x), the Gaussian factors, and conj(psi0) psi
      constexpr int ISTEP = 256 >> SH::logC;
      const int l = tid & (C - 1), i0 = tid >> logC;
      const bool ph = !OBS || (f & F_PHASE);
      LineRec<T> rec;
      if (ph) rec = sRec[l];
      const T* G0 = p.G[0][p.axis];
      const T* G1 = p.G[1][p.axis];
      // global index of point k of this thread: gbase + k gstep (autocorrelation)
      [[maybe_unused]] int64_t gbase = 0, gstep = 0;
      if constexpr (OBS && !GRID) {
        if (f & F_AUTOCORR) {
          int ll, ii;
          int64_t es;
          fixed_walk<T, SH>(p, o0, cb, ll, ii, gbase, es);
          gstep = es * ISTEP;
        }
      }
      const bool g0 = ph && p.ngauss > 0 && gauss_line_active(rec.g[0]);
      const bool g1 = ph && p.ngauss > 1 && gauss_line_active(rec.g[1]);
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int i = i0 + k * ISTEP;
        cx<T> v = s[i * LS + l];
        if (ph) {
          // without additive terms the factors are exactly 1 and the product is skipped
          if (p.sep) v = apply_factor_rec(v, p.Prec[i], rec.L);
          if (g0) v = apply_gauss_phase(v, rec.g[0] * G0[i]);
          if (g1) v = apply_gauss_phase(v, rec.g[1] * G1[i]);
          s[i * LS + l] = v;
        }
        if constexpr (OBS) {
          if (f & F_OBS_POS) {
            const T rho = norm2(v);
            const cx<T> xx = p.Ox[i];
            q[0] = q[0] + rho;
            q[1] = madd(xx.re, rho, q[1]);
            q[2] = madd(xx.im, rho, q[2]);
            q[3] = madd(p.AT[i], rho, q[3]);
            if (p.ngauss > 0) q[4] = madd(G0[i], rho, q[4]);
            if (p.ngauss > 1) q[5] = madd(G1[i], rho, q[5]);
            if (!GRID && (f & F_AUTOCORR)) {  // GRID: after the grid phase, below
              const cx<T> c = cmulc(v, p.psi0[gbase + k * gstep]);
              q[6] = q[6] + c.re;
              q[7] = q[7] + c.im;
            }
          }
        }
      }
      // static grid potential (GRID variant only): its phase records and its
      // potential-energy sum
      if constexpr (GRID) {
        int ll, ii;
        int64_t gb, es;
        fixed_walk<T, SH>(p, o0, cb, ll, ii, gb, es);
        const int64_t gs = es * ISTEP;
        const bool gph = ph && p.grid_rec != nullptr;
#pragma unroll
        for (int k = 0; k < 8; k++) {
          const int i = i0 + k * ISTEP;
          cx<T> v = s[i * LS + l];
          if (gph) {
            v = tw_apply<false>(v, p.grid_rec[gb + k * gs]);
            s[i * LS + l] = v;
          }
          if constexpr (OBS) {
            if (f & F_OBS_POS) {
              if (p.grid_v) q[3] = madd(T(p.grid_v[gb + k * gs]), norm2(v), q[3]);
              if (f & F_AUTOCORR) {
                const cx<T> c = cmulc(v, p.psi0[gb + k * gs]);
                q[6] = q[6] + c.re;
                q[7] = q[7] + c.im;
              }
            }
          }
        }
      }
    } else {
    for (int e = tid; e < ntot; e += nthr) {
      const int l = e & (C - 1), i = e >> logC;
      cx<T> v = s[i * LS + l];
      if (f & F_PHASE) {
        if (p.sep) v = apply_factor(v, Pa[i], Pal[i], sLh[l], sLl[l]);
        for (int gg = 0; gg < p.ngauss; gg++) v = apply_gauss_phase(v, sGl[gg][l] * p.G[gg][p.axis][i]);
        if (p.grid_rec) v = tw_apply<false>(v, p.grid_rec[tile_gidx(p, sh, o0, cb, i, l)]);
        s[i * LS + l] = v;
      }
      if (OBS && (f & F_OBS_POS)) {
        int gi[3];
        if (contig)
          grid_index(p.g, p.axis, o0 + l, 0, i, gi);
        else
          grid_index(p.g, p.axis, o0, cb + l, i, gi);
        const double re = (double)v.re, im = (double)v.im;
        const double rho = re * re + im * im;
        acc[Q_RHO] += rho;
        double V = 0.0;
        for (int d = 0; d < p.g.ndim; d++) {
          const double x = p.g.xmin[d] + (double)gi[d] * p.g.dx[d];
          acc[Q_X + d] += x * rho;
          acc[Q_XX + d] += x * x * rho;
          V += p.A[d][gi[d]];
        }
        for (int gg = 0; gg < p.ngauss; gg++) {
          double prod = p.ctrl->gcoef[gg];
          for (int d = 0; d < p.g.ndim; d++) prod *= p.Gd[gg][d][gi[d]];
          V += prod;
        }
        if (p.grid_v) V += p.grid_v[tile_gidx(p, sh, o0, cb, i, l)];
        acc[Q_V] += V * rho;
        if (f & F_AUTOCORR) {
          const cx<T> z = p.psi0[tile_gidx(p, sh, o0, cb, i, l)];
          acc[Q_AC_RE] += (double)z.re * re + (double)z.im * im;
          acc[Q_AC_IM] += (double)z.re * im - (double)z.im * re;
        }
      }
    }
    }
    __syncthreads();
  }

  if (f & (F_FFT | F_KIN)) tile_fft<T, E, false>(s, p, sh, tid);

  if (f & ((OBS ? F_OBS_MOM : 0u) | F_KIN)) {
    if (f & F_KIN) {
      if constexpr (SH::fixed) {
        for (int l = tid; l < C; l += nthr) sRec[l] = p.lines_kin[contig ? o0 + l : cb + l];
      } else {
        line_factors<T>(p, p.K, p.K_lo, false, contig, o0, cb, C, sLh, sLl, sGl);
      }
      __syncthreads();
    }
    const cx<T>* Ka = p.K[p.axis];
    const cx<T>* Kal = p.K_lo[p.axis];
    if constexpr (SH::fixed) {
      // with OBS: the thread's line sums of |psi_hat|^2 times 1, k, k^2
      constexpr int ISTEP = 256 >> SH::logC;
      const int l = tid & (C - 1), i0 = tid >> logC;
      const bool kin = !OBS || (f & F_KIN);
      TwE<T> L;
      if (kin) L = sRec[l].L;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int i = i0 + k * ISTEP;
        if constexpr (OBS) {
          if (f & F_OBS_MOM) {
            const T rho = norm2(s[i * LS + l]);
            const cx<T> kk = p.Ok[i];
            q[0] = q[0] + rho;
            q[1] = madd(kk.re, rho, q[1]);
            q[2] = madd(kk.im, rho, q[2]);
          }
        }
        if (kin) s[i * LS + l] = apply_factor_rec(s[i * LS + l], p.Krec[i], L);
      }
    } else {
    for (int e = tid; e < ntot; e += nthr) {
      const int l = e & (C - 1), i = e >> logC;
      cx<T> v = s[i * LS + l];
      if (OBS && (f & F_OBS_MOM)) {
        int gi[3];
        if (contig)
          grid_index(p.g, p.axis, o0 + l, 0, i, gi);
        else
          grid_index(p.g, p.axis, o0, cb + l, i, gi);
        const double re = (double)v.re, im = (double)v.im;
        const double rho = re * re + im * im;
        acc[Q_RHOK] += rho;
        for (int d = 0; d < p.g.ndim; d++) {
          const double k = wavenumber(p.g, d, gi[d]);
          acc[Q_K + d] += k * rho;
          acc[Q_K2] += k * k * rho;
        }
      }
      if (f & F_KIN) s[i * LS + l] = apply_factor(v, Ka[i], Kal[i], sLh[l], sLl[l]);
    }
    }
    __syncthreads();
    if (f & F_KIN) tile_fft<T, E, true>(s, p, sh, tid);
  }

  if (!(f & F_NO_STORE)) {
    if constexpr (SH::fixed) {
      constexpr int ISTEP = 256 >> SH::logC;
      int l, i0;
      int64_t base, es;
      fixed_walk<T, SH>(p, o0, cb, l, i0, base, es);
      cx<T>* dst = p.out + base;
      const int64_t step = es * ISTEP;
#pragma unroll
      for (int k = 0; k < 8; k++) dst[k * step] = s[(i0 + k * ISTEP) * LS + l];
    } else {
      for (int e = tid; e < ntot; e += nthr) {
        const int i = e >> logC, l = e & (C - 1);
        p.out[tile_gidx(p, sh, o0, cb, i, l)] = s[i * LS + l];
      }
    }
  }

  if (OBS && (f & (F_OBS_POS | F_OBS_MOM))) {
    if constexpr (SH::fixed) {
      __syncthreads();  // the tile is free now: it holds the per-warp line sums
      fixed_obs_reduce<T, SH>(p, q, o0, cb, reinterpret_cast<T*>(s), red);
    } else {
      block_sum(acc, tot, red);
      if (tid < NQ) p.partials[blockIdx.x * (int64_t)NQ + tid] = tot[tid];
    }
  }
  __syncthreads();
}

// One tile per block: synchronous load, then compute.
template <class T, int E, bool OBS, class SH, bool GRID = false>
__device__ __forceinline__ void pass_body(const PassParams<T>& p, const SH& sh, cx<T>* s) {
  const int64_t tile = blockIdx.x;
  if constexpr (SH::fixed) {
    fixed_load<T, SH>(p, s, tile);
  } else {
    int64_t o0, cb;
    tile_origin(p, sh, tile, o0, cb);
    const int C = 1 << sh.logC, ntot = C << sh.logn;
    for (int e = threadIdx.x; e < ntot; e += sh.nthr) {
      const int i = e >> sh.logC, l = e & (C - 1);
      s[i * sh.LS + l] = p.in[tile_gidx(p, sh, o0, cb, i, l)];
    }
  }
  __syncthreads();
  pass_compute<T, E, OBS, SH, GRID>(p, sh, s, tile);
}

// E elements per thread; the block has at most 32 E threads, so a tile holds at most
// 32 E^2 elements (2048 for E = 8, 8192 for E = 16). OBS compiles the partial sums in.
template <class T, int E, bool OBS>
__global__ void __launch_bounds__(32 * E) k_pass(const PassParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_body<T, E, OBS>(p, DynShape(p), reinterpret_cast<cx<T>*>(smem_raw));
}

// Batched pass over the instances of one shape class: block b of the launch is block
// block_off + b of the class-sorted block list (tile_start[k]: first block of instance k),
// serving tile (block - tile_start[inst]) of instance block_inst[block]. Every instance
// tiles its lines into 2048-element tiles with 256 threads. The block copies its
// instance's parameters to shared memory and runs the pass body: LOGN = 6..10 the
// compile-time-shape body (with per-line records), LOGN = 0 the run-time one.
// raw: a 16-byte aligned shared-memory buffer of sizeof(PassParams<T>) bytes for the
// instance's parameters (the caller's, so that several bodies in one kernel share it).
template <class T, bool CONTIG, int LOGN>
__device__ __forceinline__ void pass_batch_body(const PassParams<T>* __restrict__ params,
                                                const int64_t* __restrict__ tile_start,
                                                const int* __restrict__ block_inst, int64_t blk, uint32_t flags,
                                                int khalf, unsigned char* raw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassParams<T>& p = *reinterpret_cast<PassParams<T>*>(raw);
  const int inst = block_inst[blk];
  const int64_t tile = blk - tile_start[inst];
  // fixed shapes: the tile loads need only the state pointer and the axis stride, so they
  // are issued before the parameter copy and the two latencies overlap
  [[maybe_unused]] cx<T> v[8];
  [[maybe_unused]] int vl = 0, vi0 = 0;
  if constexpr (LOGN > 0) {
    using SH = FixShape<LOGN, CONTIG>;
    constexpr int ISTEP = 256 >> SH::logC;
    const cx<T>* in = params[inst].in;
    const int li = params[inst].log_inner;
    vl = threadIdx.x & ((1 << SH::logC) - 1);
    vi0 = threadIdx.x >> SH::logC;
    int64_t base, es;
    if (CONTIG) {
      base = (((tile << SH::logC) + vl) << SH::logn) + vi0;
      es = 1;
    } else {
      const int tpo = li - SH::logC;
      const int64_t o0 = tile >> tpo, cb = (tile & ((int64_t(1) << tpo) - 1)) << SH::logC;
      es = int64_t(1) << li;
      base = (((o0 << SH::logn) + vi0) << li) + cb + vl;
    }
    const cx<T>* q = in + base;
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = q[k * es * ISTEP];
  }
  const int* src = reinterpret_cast<const int*>(&params[inst]);
  for (int k = threadIdx.x; k < (int)(sizeof(PassParams<T>) / sizeof(int)); k += blockDim.x)
    reinterpret_cast<int*>(raw)[k] = src[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    p.flags = flags;
    if (khalf) {
      for (int d = 0; d < 3; d++) {
        p.K[d] = p.Khalf_axes[d];
        p.K_lo[d] = p.Khalf_lo_axes[d];
      }
      p.Krec = p.Krec_half;
      p.lines_kin = p.lines_kin_half;
    }
  }
  __syncthreads();
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  if constexpr (LOGN > 0) {
    using SH = FixShape<LOGN, CONTIG>;
    constexpr int ISTEP = 256 >> SH::logC;
#pragma unroll
    for (int k = 0; k < 8; k++) s[(vi0 + k * ISTEP) * SH::LS + vl] = v[k];
    __syncthreads();
    pass_compute<T, 8, false>(p, SH(), s, tile);
  } else {
    const DynShape sh(p);
    int64_t o0, cb;
    tile_origin(p, sh, tile, o0, cb);
    const int C = 1 << sh.logC, ntot = C << sh.logn;
    for (int e = threadIdx.x; e < ntot; e += sh.nthr) {
      const int i = e >> sh.logC, l = e & (C - 1);
      s[i * sh.LS + l] = p.in[tile_gidx(p, sh, o0, cb, i, l)];
    }
    __syncthreads();
    pass_compute<T, 8, false>(p, sh, s, tile);
  }
}

template <class T, bool CONTIG, int LOGN>
__global__ void __launch_bounds__(256) k_pass_batch(const PassParams<T>* __restrict__ params,
                                                    const int64_t* __restrict__ tile_start,
                                                    const int* __restrict__ block_inst, int64_t block_off,
                                                    uint32_t flags, int khalf) {
  __shared__ __align__(16) unsigned char raw[sizeof(PassParams<T>)];
  pass_batch_body<T, CONTIG, LOGN>(params, tile_start, block_inst, block_off + blockIdx.x, flags, khalf, raw);
}
// FP64 with a compile-time shape (LOGN = 6..10): at most 64 registers, so that four
// blocks share an SM (the FP64 pipe needs the warps to cover its latency).
template <bool CONTIG, int LOGN>
__global__ void __launch_bounds__(256, 4) k_pass_batch_f64(const PassParams<double>* __restrict__ params,
                                                          const int64_t* __restrict__ tile_start,
                                                          const int* __restrict__ block_inst, int64_t block_off,
                                                          uint32_t flags, int khalf) {
  __shared__ __align__(16) unsigned char raw[sizeof(PassParams<double>)];
  pass_batch_body<double, CONTIG, LOGN>(params, tile_start, block_inst, block_off + blockIdx.x, flags, khalf, raw);
}

template <class T>
__device__ void lines_body(const LinesParams<T>& p, int64_t first, int64_t stride);

// Batched per-line records: blockIdx.y selects the instance, x strides over its lines.
template <class T>
__global__ void __launch_bounds__(256) k_lines_batch(const LinesParams<T>* __restrict__ params) {
  __shared__ __align__(16) unsigned char raw[sizeof(LinesParams<T>)];
  const int* src = reinterpret_cast<const int*>(&params[blockIdx.y]);
  for (int k = threadIdx.x; k < (int)(sizeof(LinesParams<T>) / sizeof(int)); k += blockDim.x)
    reinterpret_cast<int*>(raw)[k] = src[k];
  __syncthreads();
  const LinesParams<T>& p = *reinterpret_cast<const LinesParams<T>*>(raw);
  lines_body<T>(p, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Fixed-size pass: n = 2^LOGN points per line, 2048-element tiles, 256 threads.
// GRID: the variant that also applies a static grid potential (contiguous passes only).
template <class T, int LOGN, bool CONTIG, bool OBS, bool GRID = false>
__global__ void __launch_bounds__(256) k_pass_fixed(const PassParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_body<T, 8, OBS, FixShape<LOGN, CONTIG>, GRID>(p, FixShape<LOGN, CONTIG>(), reinterpret_cast<cx<T>*>(smem_raw));
}
// FP64: at most 64 registers, so that four blocks share an SM (the FP64 pipe needs the
// warps to cover its latency); the passes that also form observable sums or apply a grid
// potential, at most 80 (three blocks).
template <int LOGN, bool CONTIG, bool OBS, bool GRID = false>
__global__ void __launch_bounds__(256, (OBS || GRID) ? 3 : 4) k_pass_fixed_f64(const PassParams<double> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_body<double, 8, OBS, FixShape<LOGN, CONTIG>, GRID>(p, FixShape<LOGN, CONTIG>(),
                                                          reinterpret_cast<cx<double>*>(smem_raw));
}

// ------------------------------------------------------------------ per-line records
// One record per line of a pass: the FP64 product of the other axes' factors (high +
// low table parts), rounded to a record, and the per-line Gaussian-term phase
// coefficients. Lines first, first + stride, ...
template <class T>
__device__ void lines_body(const LinesParams<T>& p, int64_t first, int64_t stride) {
  const bool contig = (p.axis == p.g.ndim - 1);
  for (int64_t line = first; line < p.nlines; line += stride) {
    int gi[3];
    if (contig)
      grid_index(p.g, p.axis, line, 0, 0, gi);
    else
      grid_index(p.g, p.axis, 0, line, 0, gi);
    double r = 1.0, m = 0.0;
    for (int d = 0; d < p.g.ndim; d++) {
      if (d == p.axis) continue;
      const cx<T> hh = p.H[d][gi[d]], ll = p.Lo[d][gi[d]];
      const double fr = (double)hh.re + (double)ll.re, fi = (double)hh.im + (double)ll.im;
      const double nr = r * fr - m * fi, ni = r * fi + m * fr;
      r = nr;
      m = ni;
    }
    LineRec<T> rec;
    rec.L = make_rec<T>(r, m);
    for (int gg = 0; gg < WP_MAX_GAUSS; gg++) {
      double prod = 0.0;
      if (p.gauss && gg < p.ngauss) {
        prod = p.ctrl->gphase[gg];
        for (int d = 0; d < p.g.ndim; d++)
          if (d != p.axis) prod *= p.Gd[gg][d][gi[d]];
      }
      rec.g[gg] = (T)prod;
    }
    p.out[line] = rec;
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_lines(const LinesParams<T> p) {
  lines_body<T>(p, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// ------------------------------------------------------------------ per-step tables
// One block. Forms t = t0 + (step + step_add) dt + t_shift, stores the new step index,
// and fills, for every axis, the additive potential A_d(x, t), its phase factor
// exp(-i A_d tau/hbar) (argument reduced by the FP64 sincos), and the Gaussian-term
// factors; the Gaussian coefficients f_g(t) and f_g(t) tau/hbar go to the control block.
template <class T>
__device__ void prep_body(const PrepParams<T>& p, int blk, int nblk) {
  __shared__ int64_t s_step;
  if (threadIdx.x == 0) s_step = p.ctrl->step + p.step_add;
  __syncthreads();
  const int64_t step = s_step;
  const double t = p.g.t0 + (double)step * p.g.dt + p.t_shift;
  const DevPot& pot = *p.pot;
  __shared__ double fco[WP_MAX_TERMS];
  if (threadIdx.x < pot.nterms) fco[threadIdx.x] = term_coef(pot.term[threadIdx.x], t);
  __syncthreads();
  [[maybe_unused]] const double tau_hbar = p.tau / p.g.hbar;
  // one flat range over the entries of all axes, so that short axes share a round
  const int64_t n01 = p.n[0] + (p.g.ndim > 1 ? p.n[1] : 0);
  const int64_t nall = n01 + (p.g.ndim > 2 ? p.n[2] : 0);
  for (int64_t e = blk * (int64_t)blockDim.x + threadIdx.x; e < nall; e += (int64_t)nblk * blockDim.x) {
    {
      const int d = e < p.n[0] ? 0 : (e < n01 ? 1 : 2);
      const int64_t i = e - (d == 0 ? 0 : (d == 1 ? p.n[0] : n01));
      const AxisTab<T>& tb = p.tab[d];
      const double x = p.g.xmin[d] + (double)i * p.g.dx[d];
      double A = 0.0;
      for (int k = 0; k < pot.nterms; k++) {
        const wp_pot_term& tm = pot.term[k];
        if (tm.shape == WP_SHAPE_GAUSS) continue;
        const double part = term_axis_part(tm, d, x, t);
        if (part != 0.0) A += fco[k] * part;
      }
      tb.A[i] = A;
      if (tb.AT) tb.AT[i] = (T)A;
      if constexpr (std::is_same<T, float>::value) {
        // complex64: the factor's high and low parts straight from the float-float cos and
        // sin of the argument (FP64 only reduces it)
        ff c, sn;
        cis_ff(-A * tau_hbar, c, sn);
        TwE<float> r;
        r.h = mk(c.hi, sn.hi);
        r.l = mk(c.lo, sn.lo);
        tb.P[i] = r.h;
        tb.P_lo[i] = r.l;
        tb.Prec[i] = r;
      } else {
        double sn, cs;
        sincos(-A * p.tau / p.g.hbar, &sn, &cs);
        const T hc = (T)cs, hs = (T)sn;
        tb.P[i] = mk(hc, hs);
        tb.P_lo[i] = mk((T)(cs - (double)hc), (T)(sn - (double)hs));
        tb.Prec[i] = make_rec<T>(cs, sn);
      }
      for (int gg = 0; gg < pot.ngauss; gg++) {
        const double gf = gauss_axis_factor(pot.term[pot.gauss_term[gg]], d, x, t);
        tb.Gd[gg][i] = gf;
        tb.G[gg][i] = (T)gf;
      }
    }
  }
  // The last block to finish publishes the Gaussian coefficients, the table time and the
  // new step index: every block has read the old index before it counts itself done.
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (nblk == 1) {
      s_last = true;
    } else {
      __threadfence();
      s_last = atomicAdd(&p.ctrl->prep_done, 1u) == (unsigned)(nblk - 1);
    }
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    for (int gg = 0; gg < WP_MAX_GAUSS; gg++) {
      double fc = 0.0;
      if (gg < pot.ngauss) fc = term_coef(pot.term[pot.gauss_term[gg]], t);
      p.ctrl->gcoef[gg] = fc;
      p.ctrl->gphase[gg] = fc * p.tau / p.g.hbar;
    }
    p.ctrl->t_tab = t;
    p.ctrl->step = step;
    if (nblk > 1) p.ctrl->prep_done = 0u;
  }
}

template <class T>
__global__ void __launch_bounds__(64) k_prep(const PrepParams<T> p) {
  prep_body<T>(p, blockIdx.x, gridDim.x);
}

// Batched tables: block b updates instance b. The step increment, the time shift and the
// phase length (in units of the instance's dt) are the same for all instances.
template <class T>
__global__ void __launch_bounds__(256) k_prep_batch(const PrepParams<T>* __restrict__ params, int step_add,
                                                    double shift_dt, double tau_dt) {
  __shared__ __align__(16) unsigned char raw[sizeof(PrepParams<T>)];
  PrepParams<T>& p = *reinterpret_cast<PrepParams<T>*>(raw);
  const int* src = reinterpret_cast<const int*>(&params[blockIdx.x]);
  for (int k = threadIdx.x; k < (int)(sizeof(PrepParams<T>) / sizeof(int)); k += blockDim.x)
    reinterpret_cast<int*>(raw)[k] = src[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    p.step_add = step_add;
    p.t_shift = shift_dt * p.g.dt;
    p.tau = tau_dt * p.g.dt;
  }
  __syncthreads();
  prep_body<T>(p, 0, 1);
}

// ------------------------------------------------------------------ 1-D resident kernel
// One CTA holds one 1-D line in shared memory for a chunk of steps: the whole step
// (potential phase, FFT, kinetic factor, inverse FFT) runs without touching HBM.
// V(x,t) = sum_k f_k(t) s_k(x,t) split by time dependence (Eq. 9 applied with the terms of
// Tab. 2): static terms come from the tables S (built once per potential), linear and
// constant terms sum to beta(t) x - gamma(t), whose phase at x_j = xmin + j dx is the
// plane wave exp(-i (theta0 + j delta)) = hiT[j / 64] loT[j mod 64] (both tables formed
// per step with FP64 sincos of directly computed arguments), and the remaining terms are
// evaluated at every point in FP64. The factors are applied one after the other as
// records (complex64: high and low parts), so that the per-point work of the common
// potentials stays off the FP64 pipe.
// Line shape of the resident kernel: Res1dDyn holds the length and block size at run
// time (E elements per thread, run-time Stockham stages); Res1dFix<LOGN, EPT> makes them
// compile-time constants (n = 2^LOGN, n / EPT threads, unrolled stages with per-stage
// twiddle records, kinetic factors as records).
template <int E>
struct Res1dDyn {
  static constexpr bool fixed = false;
  int logn, n, nthr;
  template <class T>
  __device__ explicit Res1dDyn(const Res1dParams<T>& p) : logn(p.logn), n(1 << p.logn), nthr(p.nthreads) {}
  template <class T, bool INV>
  __device__ __forceinline__ void fft(cx<T>* s, const Res1dParams<T>& p, int tid) const {
    fft_tile<T, E, INV>(s, logn, 0, 1, p.W, p.W_lo, tid, nthr, p.max_radix_log);
  }
};

template <int LOGN, int EPT>
struct Res1dFix {
  static constexpr bool fixed = true;
  static constexpr int logn = LOGN, n = 1 << LOGN, nthr = (1 << LOGN) / EPT;
  template <class T>
  __device__ explicit Res1dFix(const Res1dParams<T>&) {}
  template <class T, bool INV>
  __device__ __forceinline__ void fft(cx<T>* s, const Res1dParams<T>& p, int tid) const {
    fft_fixed<T, LOGN, 0, 1, INV, 0, EPT, false>(s, reinterpret_cast<const TwE<T>*>(p.Wst), tid);
  }
};

template <class T, class RS>
__device__ void res1d_potential_phase(cx<T>* s, const Res1dParams<T>& p, const RS& rs, double t, int half,
                                      double* fco, TwE<T>* hiT, TwE<T>* loT, int tid) {
  const DevPot& pot = *p.pot;
  const double tau = half ? 0.5 * p.g.dt : p.g.dt;
  const int n = rs.n, nthr = rs.nthr;
  __syncthreads();
  if (tid < pot.nterms) fco[tid] = term_coef(pot.term[tid], t);
  __syncthreads();
  const bool plane = p.plane_mask != 0;
  if (plane) {
    double beta = 0.0, gamma = 0.0;
    for (int k = 0; k < pot.nterms; k++) {
      if (!((p.plane_mask >> k) & 1u)) continue;
      const wp_pot_term& tm = pot.term[k];
      if (tm.shape == WP_SHAPE_LINEAR) {
        beta += fco[k] * tm.a[0];
        gamma += fco[k] * tm.a[0] * (tm.c0[0] + tm.v[0] * t);
      } else {
        gamma -= fco[k];
      }
    }
    const double th0 = tau * (beta * p.g.xmin[0] - gamma) / p.g.hbar;
    const double del = tau * beta * p.g.dx[0] / p.g.hbar;
    const int nhi = n > 64 ? n >> 6 : 1, nlo = n < 64 ? n : 64;
    for (int k = tid; k < nhi + nlo; k += nthr) {
      double sn, cs;
      if (k < nhi) {
        sincos(-fma((double)(k << 6), del, th0), &sn, &cs);
        hiT[k] = make_rec<T>(cs, sn);
      } else {
        sincos(-(double)(k - nhi) * del, &sn, &cs);
        loT[k - nhi] = make_rec<T>(cs, sn);
      }
    }
    __syncthreads();
  }
  const TwE<T>* S = p.S[half ? 1 : 0];
  const bool stat = p.static_mask != 0;
  for (int i = tid; i < n; i += nthr) {
    cx<T> v = s[i];
    if (stat) v = tw_apply<false>(v, S[i]);
    if (plane) {
      v = tw_apply<false>(v, hiT[i >> 6]);
      v = tw_apply<false>(v, loT[i & 63]);
    }
    if (p.gen_mask) {
      const double x = p.g.xmin[0] + (double)i * p.g.dx[0];
      double V = 0.0;
      for (int k = 0; k < pot.nterms; k++) {
        if (!((p.gen_mask >> k) & 1u)) continue;
        const wp_pot_term& tm = pot.term[k];
        const double sh = (tm.shape == WP_SHAPE_GAUSS) ? gauss_axis_factor(tm, 0, x, t) : term_axis_part(tm, 0, x, t);
        V += fco[k] * sh;
      }
      double sn, cs;
      sincos(-V * tau / p.g.hbar, &sn, &cs);
      v = tw_apply<false>(v, make_rec<T>(cs, sn));
    }
    s[i] = v;
  }
  __syncthreads();
}

template <class T, class RS>
__device__ void res1d_kinetic(cx<T>* s, const Res1dParams<T>& p, const RS& rs, int half, int tid) {
  rs.template fft<T, false>(s, p, tid);
  if constexpr (RS::fixed) {
    const TwE<T>* K = p.Krec[half];
#pragma unroll
    for (int i = tid; i < rs.n; i += rs.nthr) s[i] = tw_apply<false>(s[i], K[i]);
  } else {
    const cx<T>* K = half ? p.Khalf : p.Kfull;
    const cx<T>* Klo = half ? p.Khalf_lo : p.Kfull_lo;
    const cx<T> one = mk((T)1, (T)0), zero = mk((T)0, (T)0);
    for (int i = tid; i < rs.n; i += rs.nthr) s[i] = apply_factor(s[i], K[i], Klo[i], one, zero);
  }
  __syncthreads();
  rs.template fft<T, true>(s, p, tid);
}

template <class T, class RS>
__device__ void res1d_body(const Res1dParams<T>& p, const RS& rs, cx<T>* s) {
  __shared__ double red[32][NQ];
  __shared__ double qp[NQ], qm[NQ];
  __shared__ double fco[WP_MAX_TERMS];
  __shared__ TwE<T> hiT[256], loT[64];  // plane-wave tables (n <= 16384)
  const int tid = threadIdx.x, nthr = rs.nthr;
  const int n = rs.n;
  const int64_t s0 = p.ctrl->step;
  const double dt = p.g.dt;
  auto tim = [&](int64_t k) { return p.g.t0 + (double)k * dt; };

  for (int i = tid; i < n; i += nthr) s[i] = p.psi[i];
  __syncthreads();

  const int64_t m = p.nsteps;
  if (m > 0) {
    if (p.order == WP_ORDER_VKV) {
      res1d_potential_phase<T>(s, p, rs, tim(s0), 1, fco, hiT, loT, tid);
      for (int64_t k = 0; k < m; k++) {
        res1d_kinetic<T>(s, p, rs, 0, tid);
        const bool last = (k == m - 1);
        res1d_potential_phase<T>(s, p, rs, tim(s0 + k + 1), last ? 1 : 0, fco, hiT, loT, tid);
      }
    } else {
      res1d_kinetic<T>(s, p, rs, 1, tid);
      for (int64_t k = 0; k < m; k++) {
        res1d_potential_phase<T>(s, p, rs, tim(s0 + k) + 0.5 * dt, 0, fco, hiT, loT, tid);
        res1d_kinetic<T>(s, p, rs, (k == m - 1) ? 1 : 0, tid);
      }
    }
  }

  for (int i = tid; i < n; i += nthr) p.psi[i] = s[i];

  if (p.obs) {
    __syncthreads();
    const DevPot& pot = *p.pot;
    const double t = tim(s0 + m);
    if (tid < pot.nterms) fco[tid] = term_coef(pot.term[tid], t);
    __syncthreads();
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) acc[q] = 0.0;
    for (int i = tid; i < n; i += nthr) {
      const double x = p.g.xmin[0] + (double)i * p.g.dx[0];
      const double re = (double)s[i].re, im = (double)s[i].im;
      const double rho = re * re + im * im;
      double V = 0.0;
      for (int k = 0; k < pot.nterms; k++) {
        const wp_pot_term& tm = pot.term[k];
        const double sh = (tm.shape == WP_SHAPE_GAUSS) ? gauss_axis_factor(tm, 0, x, t) : term_axis_part(tm, 0, x, t);
        V += fco[k] * sh;
      }
      if (p.vgrid) V += p.vgrid[i];
      acc[Q_RHO] += rho;
      acc[Q_X] += x * rho;
      acc[Q_XX] += x * x * rho;
      acc[Q_V] += V * rho;
      if (p.autocorr) {
        const cx<T> z = p.psi0[i];
        acc[Q_AC_RE] += (double)z.re * re + (double)z.im * im;
        acc[Q_AC_IM] += (double)z.re * im - (double)z.im * re;
      }
    }
    block_sum(acc, qp, red);
    rs.template fft<T, false>(s, p, tid);
#pragma unroll
    for (int q = 0; q < NQ; q++) acc[q] = 0.0;
    for (int i = tid; i < n; i += nthr) {
      const double re = (double)s[i].re, im = (double)s[i].im;
      const double rho = re * re + im * im;
      const double k = wavenumber(p.g, 0, i);
      acc[Q_RHOK] += rho;
      acc[Q_K] += k * rho;
      acc[Q_K2] += k * k * rho;
    }
    block_sum(acc, qm, red);
    if (tid == 0) {
      const int64_t slot = p.ctrl->nobs;
      if (slot < p.obs_cap) {
        finish_obs(qp, qm, p.g, n, p.autocorr, t, s0 + m, p.obs_out + slot * 16);
        if (!isfinite(p.obs_out[slot * 16 + 1])) p.ctrl->err = WP_ENONFINITE;
      }
      p.ctrl->nobs = slot + 1;
    }
  }
  if (tid == 0) p.ctrl->step = s0 + m;
}

template <class T, int E, int MAXT>
__global__ void __launch_bounds__(MAXT) k_res1d(const Res1dParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  res1d_body<T>(p, Res1dDyn<E>(p), reinterpret_cast<cx<T>*>(smem_raw));
}

// Fixed-length resident line: n = 2^LOGN, n / EPT threads.
template <class T, int LOGN, int EPT>
__global__ void __launch_bounds__((1 << LOGN) / EPT) k_res1d_fixed(const Res1dParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  res1d_body<T>(p, Res1dFix<LOGN, EPT>(p), reinterpret_cast<cx<T>*>(smem_raw));
}

// Static phase tables: exp(-i V_s(x_j) tau / hbar) for tau = dt and dt/2, V_s the sum of
// the static terms (time-independent coefficient and centre) of a 1-D potential, formed
// in FP64 and stored as records of T.
template <class T>
__global__ void __launch_bounds__(256) k_static_phase(const StaticPhaseParams<T> p) {
  const DevPot& pot = *p.pot;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = p.g.xmin[0] + (double)i * p.g.dx[0];
    double V = 0.0;
    for (int k = 0; k < pot.nterms; k++) {
      if (!((p.static_mask >> k) & 1u)) continue;
      const wp_pot_term& tm = pot.term[k];
      const double sh = (tm.shape == WP_SHAPE_GAUSS) ? gauss_axis_factor(tm, 0, x, 0.0) : term_axis_part(tm, 0, x, 0.0);
      V += term_coef(tm, 0.0) * sh;
    }
    if (p.vgrid) V += p.vgrid[i];
    double sn, cs;
    sincos(-V * p.g.dt / p.g.hbar, &sn, &cs);
    p.S[0][i] = make_rec<T>(cs, sn);
    sincos(-V * (0.5 * p.g.dt) / p.g.hbar, &sn, &cs);
    p.S[1][i] = make_rec<T>(cs, sn);
  }
}

// Phase records exp(-i V_j tau / hbar) of a static grid potential for tau = dt and dt/2
// (FP64 sincos, stored as records of T).
template <class T>
__global__ void __launch_bounds__(256) k_grid_phase(const GridPhaseParams<T> p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double V = p.V[i];
    double sn, cs;
    sincos(-V * p.dt / p.hbar, &sn, &cs);
    p.rec[0][i] = make_rec<T>(cs, sn);
    sincos(-V * (0.5 * p.dt) / p.hbar, &sn, &cs);
    p.rec[1][i] = make_rec<T>(cs, sn);
  }
}

// User expectation value <psi|A|psi> (Sec. 3.2.5): per-block FP64 sums over a fixed
// range of points, then one block sums the partials in order.
template <class T>
__global__ void __launch_bounds__(256) k_expect_partial(const ExpectParams<T> p) {
  __shared__ double red[32][NQ];
  __shared__ double tot[NQ];
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) acc[q] = 0.0;
  const int64_t b0 = (int64_t)blockIdx.x * p.per_block;
  const int64_t b1 = b0 + p.per_block < p.n ? b0 + p.per_block : p.n;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const cx<T> v = p.psi[i];
    const double re = (double)v.re, im = (double)v.im;
    acc[0] += p.A[i] * (re * re + im * im);
  }
  block_sum(acc, tot, red);
  if (threadIdx.x == 0) p.partial[blockIdx.x] = tot[0];
}

template <class T>
__global__ void __launch_bounds__(256) k_expect_final(const double* partial, int nblocks, double dv, double* out) {
  __shared__ double red[32][NQ];
  __shared__ double tot[NQ];
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) acc[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc[0] += partial[b];
  block_sum(acc, tot, red);
  if (threadIdx.x == 0) *out = tot[0] * dv;
}

// Batched resident lines: block b runs instance b (all of one line length) for nsteps.
template <class T, class RS>
__device__ __forceinline__ void res1d_batch_body(const Res1dParams<T>* __restrict__ params, int64_t nsteps,
                                                 cx<T>* s) {
  __shared__ __align__(16) unsigned char raw[sizeof(Res1dParams<T>)];
  Res1dParams<T>& p = *reinterpret_cast<Res1dParams<T>*>(raw);
  const int* src = reinterpret_cast<const int*>(&params[blockIdx.x]);
  for (int k = threadIdx.x; k < (int)(sizeof(Res1dParams<T>) / sizeof(int)); k += blockDim.x)
    reinterpret_cast<int*>(raw)[k] = src[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    p.nsteps = nsteps;
    p.obs = 0;
  }
  __syncthreads();
  res1d_body<T>(p, RS(p), s);
}

template <class T, int E, int MAXT>
__global__ void __launch_bounds__(MAXT) k_res1d_batch(const Res1dParams<T>* __restrict__ params, int64_t nsteps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  res1d_batch_body<T, Res1dDyn<E>>(params, nsteps, reinterpret_cast<cx<T>*>(smem_raw));
}

template <class T, int LOGN, int EPT>
__global__ void __launch_bounds__((1 << LOGN) / EPT)
    k_res1d_fixed_batch(const Res1dParams<T>* __restrict__ params, int64_t nsteps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  res1d_batch_body<T, Res1dFix<LOGN, EPT>>(params, nsteps, reinterpret_cast<cx<T>*>(smem_raw));
}

#ifdef WP_COMMON_KERNELS
// ------------------------------------------------------------------ reduction kernel
// First level: block (b, y) sums rows [b R, b R + R) of the position (y = 0) or momentum
// (y = 1) partials in a fixed order and leaves the sum in row b R, which no other block
// reads. The sums are then in rows 0, R, 2R, ... (the partials are scratch of one record).
__global__ void __launch_bounds__(256) k_reduce_rows(double* pos, int64_t npos, double* mom, int64_t nmom,
                                                     int64_t R) {
  __shared__ double red[32][NQ];
  __shared__ double tot[NQ];
  double* a = blockIdx.y ? mom : pos;
  const int64_t n = blockIdx.y ? nmom : npos;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  if (r0 >= n) return;  // the whole block leaves
  const int64_t r1 = r0 + R < n ? r0 + R : n;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) acc[q] = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double2* row = reinterpret_cast<const double2*>(a + r * NQ);
#pragma unroll
    for (int q = 0; q < NQ / 2; q++) {
      const double2 v = row[q];
      acc[2 * q] += v.x;
      acc[2 * q + 1] += v.y;
    }
  }
  block_sum(acc, tot, red);  // every thread has read its rows before the first barrier in it
  if (threadIdx.x < NQ) a[r0 * NQ + threadIdx.x] = tot[threadIdx.x];
}

// One block: sums the (first-level) partials in a fixed order and writes the observable
// record.
__global__ void __launch_bounds__(256) k_reduce(const ReduceParams p) {
  __shared__ double red[32][NQ];
  __shared__ double qp[NQ], qm[NQ];
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) acc[q] = 0.0;
  for (int64_t r = threadIdx.x; r < p.npos; r += blockDim.x)
#pragma unroll
    for (int q = 0; q < NQ; q++) acc[q] += p.pos[r * p.pos_stride * NQ + q];
  block_sum(acc, qp, red);
#pragma unroll
  for (int q = 0; q < NQ; q++) acc[q] = 0.0;
  for (int64_t r = threadIdx.x; r < p.nmom; r += blockDim.x)
#pragma unroll
    for (int q = 0; q < NQ; q++) acc[q] += p.mom[r * p.mom_stride * NQ + q];
  block_sum(acc, qm, red);
  if (threadIdx.x == 0) {
    const int64_t slot = p.ctrl->nobs;
    if (slot < p.obs_cap) {
      finish_obs(qp, qm, p.g, p.ntotal, p.autocorr, p.ctrl->t_tab, p.ctrl->step, p.obs_out + slot * 16);
      if (!isfinite(p.obs_out[slot * 16 + 1])) p.ctrl->err = WP_ENONFINITE;
    }
    p.ctrl->nobs = slot + 1;
  }
}

__global__ void k_set_step(Ctrl* c, int64_t step) {
  c->step = step;
  c->nobs = 0;
  c->err = 0;
}

__global__ void k_add_step(Ctrl* c, int64_t add) { c->step += add; }
#endif  // WP_COMMON_KERNELS

// ------------------------------------------------------------------ small kernels
template <class T>
__global__ void k_convert(const ConvParams<T> p) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  if (p.dir == 0) {
    const double2 v = reinterpret_cast<const double2*>(p.src)[i];
    reinterpret_cast<cx<T>*>(p.dst)[i] = mk((T)v.x, (T)v.y);
  } else {
    const cx<T> v = reinterpret_cast<const cx<T>*>(p.src)[i];
    reinterpret_cast<double2*>(p.dst)[i] = make_double2((double)v.re, (double)v.im);
  }
}

// Normalised Gaussian packet of Sec. 4.2: a product over the axes of
// exp(-(x_d - x0_d)^2 / sigma_d^2) exp(i p0_d (x_d - x0_d) / hbar), times the normalisation.
// k_gaussian_axes forms the per-axis factors in FP64 (the normalisation folded into axis
// 0); k_gaussian multiplies them at every point.
template <class T>
__global__ void k_gaussian_axes(const GaussParams<T> p) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p.nsum; k += (int64_t)gridDim.x * blockDim.x) {
    int d = 0;
    while (d + 1 < p.g.ndim && k >= p.off[d + 1]) d++;
    const int64_t i = k - p.off[d];
    const double u = p.g.xmin[d] + (double)i * p.g.dx[d] - p.x0[d];
    double amp = exp(-u * u / (p.sigma[d] * p.sigma[d]));
    if (d == 0) amp *= p.pref;
    double sn, cs;
    sincos(p.p0[d] * u / p.g.hbar, &sn, &cs);
    p.tab[k] = mk(amp * cs, amp * sn);
  }
}

template <class T>
__global__ void k_gaussian(const GaussParams<T> p, int64_t ntotal) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ntotal) return;
  int gi[3] = {0, 0, 0};
  int64_t r = idx;
  for (int d = p.g.ndim - 1; d >= 0; d--) {
    gi[d] = (int)(r & ((1 << p.g.ln[d]) - 1));
    r >>= p.g.ln[d];
  }
  cx<double> v = p.tab[gi[0]];
  for (int d = 1; d < p.g.ndim; d++) v = cmul(v, p.tab[p.off[d] + gi[d]]);
  p.psi[idx] = mk((T)v.re, (T)v.im);
}

}  // namespace wp
