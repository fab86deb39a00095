// FP64 Stockham butterflies in fused multiply-add form, for the fixed-size transforms of
// the complex128 path (the Fourier transforms of eq. (ft), Sec. 2.1, and Algorithm 1 of
// arXiv:1306.3247).
//
// GB300 runs FP64 at 1/58 of its FP32 rate, so the complex128 passes are bound by the
// FP64 pipe, where an add costs as much as a fused multiply-add. A twiddled butterfly
// written as complex products followed by sums spends most of its slots on plain adds.
// Here every twiddle w = exp(i theta) is held in scaled form (the cosine-factor method of
// Linzer and Feig, "Implementation of efficient FFT algorithms on fused multiply-add
// architectures", IEEE Trans. Signal Process. 41 (1993)):
//
//   f = |sin theta| > |cos theta|,  s = f ? sin : cos,  t = f ? cos/sin : sin/cos (|t| <= 1)
//   (a, b) = f ? (x.im, x.re) : (x.re, x.im),  y = (a - t b, b + t a)
//   x w = (S_re y.re, S_im y.im)  with  S_re = f ? -s : s,  S_im = s
//
// so the twiddle product costs two FMAs, and the real scales S of the inputs that a
// butterfly sums are folded into the sums as FMA coefficients (ratios of two scales,
// which lie in [1/sqrt(2), sqrt(2)] in magnitude). A radix-8 butterfly takes 66 FP64
// instructions instead of 84, a radix-4 one 22 instead of 28, and the untwiddled
// radix-8 butterfly of the first stage 52 instead of 56.
//
// The records are built on the host (wp_fma_build_tables) once per axis; the same
// functions compile for the device and, with __host__/__device__ defined empty, as plain
// C++, which is how the CPU tests check them against a reference FFT.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "wp_internal.h"

#ifndef WP_HD
#define WP_HD __host__ __device__ __forceinline__
#endif

namespace wp {

// Records of one butterfly (index jm of a stage of span Ns and radix R); twiddle r
// (r = 1..R-1) is w^(r jm) with w = exp(-+ 2 pi i / (Ns R)). Bit r-1 of `flags` is f of
// twiddle r. Scales of twiddle r are S_r = (S_r.re, S_r.im); products of scales and
// ratios act component by component.
struct alignas(16) Fma2 {
  double t;        // t of w1
  int64_t flags;
  double S[2];     // S_1
};
struct alignas(16) Fma4 {
  double t[3];     // t of w1, w2, w3
  int64_t flags;
  double S2[2];    // S_2
  double S1[2];    // S_1
  double R13[2];   // S_3 / S_1
};
struct alignas(16) Fma8 {
  double t[7];     // t of w1 .. w7
  int64_t flags;
  double S4[2];    // S_4
  double S2[2];    // S_2
  double R26[2];   // S_6 / S_2
  double R15[2];   // S_5 / S_1
  double R37[2];   // S_7 / S_3
  double R13[2];   // S_3 / S_1
  double M[2];     // S_3.re / S_1.im, S_3.im / S_1.re
  double S1[2];    // S_1
  double h1;       // S_1.im / sqrt(2)
  double sg1;      // S_1.re / S_1.im (+-1)
};
static_assert(sizeof(Fma2) == 32 && sizeof(Fma4) == 80 && sizeof(Fma8) == 208, "record layout");

__host__ __device__ constexpr int wp_fma_rec_bytes(int lr) { return lr == 3 ? 208 : (lr == 2 ? 80 : 32); }
// Byte offset of the records of the stage at span 2^logNs within one direction's table
// (Ns records per stage, none for the first stage).
__host__ __device__ constexpr int wp_fma_stage_offset(int logn, int logNs) {
  int off = 0, ls = 0;
  while (ls < logNs) {
    const int lr = wp_stage_radix_log(logn, ls);
    if (ls > 0) off += (1 << ls) * wp_fma_rec_bytes(lr);
    ls += lr;
  }
  return off;
}
// Bytes of one direction's table; the forward records come first, the inverse ones
// (twiddles conjugated) follow.
__host__ __device__ constexpr int wp_fma_dir_bytes(int logn) { return wp_fma_stage_offset(logn, logn); }

// y with x w = S (.) y (see the header comment)
WP_HD cx<double> fma_tw(cx<double> x, double t, bool f) {
  const double a = f ? x.im : x.re, b = f ? x.re : x.im;
  cx<double> y;
  y.re = fma(-t, b, a);
  y.im = fma(t, a, b);
  return y;
}
WP_HD cx<double> cxd(double re, double im) {
  cx<double> r;
  r.re = re;
  r.im = im;
  return r;
}
// a + c (.) y and a - c (.) y
WP_HD cx<double> fadd(cx<double> a, const double* c, cx<double> y) {
  return cxd(fma(c[0], y.re, a.re), fma(c[1], y.im, a.im));
}
WP_HD cx<double> fsub(cx<double> a, const double* c, cx<double> y) {
  return cxd(fma(-c[0], y.re, a.re), fma(-c[1], y.im, a.im));
}
// a + rho(c (.) y) with rho = multiplication by -i (forward) or +i (inverse), and a - ...
template <bool INV>
WP_HD cx<double> fadd_rot(cx<double> a, const double* c, cx<double> y) {
  return INV ? cxd(fma(-c[1], y.im, a.re), fma(c[0], y.re, a.im)) : cxd(fma(c[1], y.im, a.re), fma(-c[0], y.re, a.im));
}
template <bool INV>
WP_HD cx<double> fsub_rot(cx<double> a, const double* c, cx<double> y) {
  return INV ? cxd(fma(c[1], y.im, a.re), fma(-c[0], y.re, a.im)) : cxd(fma(-c[1], y.im, a.re), fma(c[0], y.re, a.im));
}

// DFT of (v0, w1 v1) in place.
template <bool INV>
WP_HD void fma_dft2(cx<double>* v, const Fma2& q) {
  const cx<double> y = fma_tw(v[1], q.t, q.flags & 1);
  const cx<double> x0 = v[0];
  v[0] = fadd(x0, q.S, y);
  v[1] = fsub(x0, q.S, y);
}

// DFT of (v0, w1 v1, w2 v2, w3 v3) in place.
template <bool INV>
WP_HD void fma_dft4(cx<double>* v, const Fma4& q) {
  const int64_t f = q.flags;
  const cx<double> y1 = fma_tw(v[1], q.t[0], f & 1), y2 = fma_tw(v[2], q.t[1], f & 2),
                   y3 = fma_tw(v[3], q.t[2], f & 4);
  const cx<double> x0 = v[0];
  const cx<double> a0 = fadd(x0, q.S2, y2), a1 = fsub(x0, q.S2, y2);  // x0 +- w2 x2
  const cx<double> b2 = fadd(y1, q.R13, y3), b3 = fsub(y1, q.R13, y3);  // (w1 x1 +- w3 x3) / S1
  v[0] = fadd(a0, q.S1, b2);
  v[2] = fsub(a0, q.S1, b2);
  v[1] = fadd_rot<INV>(a1, q.S1, b3);
  v[3] = fsub_rot<INV>(a1, q.S1, b3);
}

// DFT of (v0, w1 v1, ..., w7 v7) in place: DFTs of the even and odd halves, combined
// with the powers of exp(-+ 2 pi i / 8).
template <bool INV>
WP_HD void fma_dft8(cx<double>* v, const Fma8& q) {
  const int64_t f = q.flags;
  cx<double> E0, E1, E2, E3;
  {
    // even half: DFT4 of (v0, w2 v2, w4 v4, w6 v6)
    const cx<double> y2 = fma_tw(v[2], q.t[1], f & 2), y4 = fma_tw(v[4], q.t[3], f & 8),
                     y6 = fma_tw(v[6], q.t[5], f & 32);
    const cx<double> x0 = v[0];
    const cx<double> a0 = fadd(x0, q.S4, y4), a1 = fsub(x0, q.S4, y4);
    const cx<double> b2 = fadd(y2, q.R26, y6), b3 = fsub(y2, q.R26, y6);
    E0 = fadd(a0, q.S2, b2);
    E2 = fsub(a0, q.S2, b2);
    E1 = fadd_rot<INV>(a1, q.S2, b3);
    E3 = fsub_rot<INV>(a1, q.S2, b3);
  }
  // odd half: DFT4 of (w1 v1, w3 v3, w5 v5, w7 v7), output k = S1 (.) qk
  const cx<double> y1 = fma_tw(v[1], q.t[0], f & 1), y3 = fma_tw(v[3], q.t[2], f & 4),
                   y5 = fma_tw(v[5], q.t[4], f & 16), y7 = fma_tw(v[7], q.t[6], f & 64);
  const cx<double> p0 = fadd(y1, q.R15, y5), p1 = fsub(y1, q.R15, y5);  // (w1 x1 +- w5 x5) / S1
  const cx<double> p2 = fadd(y3, q.R37, y7), p3 = fsub(y3, q.R37, y7);  // (w3 x3 +- w7 x7) / S3
  const cx<double> q0 = fadd(p0, q.R13, p2), q2 = fsub(p0, q.R13, p2);
  const cx<double> q1 = fadd_rot<INV>(p1, q.M, p3), q3 = fsub_rot<INV>(p1, q.M, p3);
  // k = 0, 4: E0 +- O0
  v[0] = fadd(E0, q.S1, q0);
  v[4] = fsub(E0, q.S1, q0);
  // k = 2, 6: E2 +- rho(O2)
  v[2] = fadd_rot<INV>(E2, q.S1, q2);
  v[6] = fsub_rot<INV>(E2, q.S1, q2);
  // k = 1, 5 and 3, 7: with O = S1.im (sg1 q.re, q.im),
  // forward  exp(-i pi/4) O = h1 (u, w),   exp(-3i pi/4) O = h1 (w', -u')
  // inverse  exp(+i pi/4) O = h1 (-w, u),  exp(+3i pi/4) O = h1 (-u', -w')
  // where u = sg1 q.re + q.im and w = q.im - sg1 q.re (u', w' of q3).
  const double u1 = fma(q.sg1, q1.re, q1.im), w1 = fma(-q.sg1, q1.re, q1.im);
  const double u3 = fma(q.sg1, q3.re, q3.im), w3 = fma(-q.sg1, q3.re, q3.im);
  const double h = q.h1;
  if (!INV) {
    v[1] = cxd(fma(h, u1, E1.re), fma(h, w1, E1.im));
    v[5] = cxd(fma(-h, u1, E1.re), fma(-h, w1, E1.im));
    v[3] = cxd(fma(h, w3, E3.re), fma(-h, u3, E3.im));
    v[7] = cxd(fma(-h, w3, E3.re), fma(h, u3, E3.im));
  } else {
    v[1] = cxd(fma(-h, w1, E1.re), fma(h, u1, E1.im));
    v[5] = cxd(fma(h, w1, E1.re), fma(-h, u1, E1.im));
    v[3] = cxd(fma(-h, u3, E3.re), fma(-h, w3, E3.im));
    v[7] = cxd(fma(h, u3, E3.re), fma(h, w3, E3.im));
  }
}

// Plain DFT4 of (x0, x1, x2, x3) into d[0..3].
template <bool INV>
WP_HD void plain_dft4(cx<double> x0, cx<double> x1, cx<double> x2, cx<double> x3, cx<double>* d) {
  const cx<double> a0 = cxd(x0.re + x2.re, x0.im + x2.im), a1 = cxd(x0.re - x2.re, x0.im - x2.im);
  const cx<double> a2 = cxd(x1.re + x3.re, x1.im + x3.im), a3 = cxd(x1.re - x3.re, x1.im - x3.im);
  d[0] = cxd(a0.re + a2.re, a0.im + a2.im);
  d[2] = cxd(a0.re - a2.re, a0.im - a2.im);
  // a1 +- rho(a3), rho = -i (forward) / +i (inverse)
  d[1] = INV ? cxd(a1.re - a3.im, a1.im + a3.re) : cxd(a1.re + a3.im, a1.im - a3.re);
  d[3] = INV ? cxd(a1.re + a3.im, a1.im - a3.re) : cxd(a1.re - a3.im, a1.im + a3.re);
}

// Untwiddled radix-8 butterfly (first stage): plain sums for the two radix-4 halves, the
// 1/sqrt(2) products of the combination folded into FMAs.
template <bool INV>
WP_HD void fma_dft8_first(cx<double>* v) {
  const double r2 = 0.707106781186547524400844362104849039;
  cx<double> e[4], o[4];
  plain_dft4<INV>(v[0], v[2], v[4], v[6], e);
  plain_dft4<INV>(v[1], v[3], v[5], v[7], o);
  v[0] = cxd(e[0].re + o[0].re, e[0].im + o[0].im);
  v[4] = cxd(e[0].re - o[0].re, e[0].im - o[0].im);
  v[2] = INV ? cxd(e[2].re - o[2].im, e[2].im + o[2].re) : cxd(e[2].re + o[2].im, e[2].im - o[2].re);
  v[6] = INV ? cxd(e[2].re + o[2].im, e[2].im - o[2].re) : cxd(e[2].re - o[2].im, e[2].im + o[2].re);
  const double u1 = o[1].re + o[1].im, w1 = o[1].im - o[1].re;
  const double u3 = o[3].re + o[3].im, w3 = o[3].im - o[3].re;
  if (!INV) {
    v[1] = cxd(fma(r2, u1, e[1].re), fma(r2, w1, e[1].im));
    v[5] = cxd(fma(-r2, u1, e[1].re), fma(-r2, w1, e[1].im));
    v[3] = cxd(fma(r2, w3, e[3].re), fma(-r2, u3, e[3].im));
    v[7] = cxd(fma(-r2, w3, e[3].re), fma(r2, u3, e[3].im));
  } else {
    v[1] = cxd(fma(-r2, w1, e[1].re), fma(r2, u1, e[1].im));
    v[5] = cxd(fma(r2, w1, e[1].re), fma(-r2, u1, e[1].im));
    v[3] = cxd(fma(-r2, u3, e[3].re), fma(-r2, w3, e[3].im));
    v[7] = cxd(fma(r2, u3, e[3].re), fma(r2, w3, e[3].im));
  }
}

// Host: fills the records of a 2^logn transform into out (2 wp_fma_dir_bytes(logn)
// bytes): forward twiddles exp(-2 pi i k / n), then inverse ones exp(+2 pi i k / n).
inline void wp_fma_build_tables(int logn, unsigned char* out) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const int dir = wp_fma_dir_bytes(logn);
  if (dir == 0) return;  // n <= 8: no twiddled stage
  memset(out, 0, 2 * (size_t)dir);
  for (int inv = 0; inv < 2; inv++) {
    int ls = 0;
    while (ls < logn) {
      const int lr = wp_stage_radix_log(logn, ls);
      const int R = 1 << lr;
      if (ls > 0) {
        unsigned char* base = out + (size_t)inv * dir + wp_fma_stage_offset(logn, ls);
        for (int jm = 0; jm < (1 << ls); jm++) {
          long double t[8] = {0}, Sre[8] = {0}, Sim[8] = {0};
          int64_t flags = 0;
          Sre[0] = Sim[0] = 1.0L;
          for (int r = 1; r < R; r++) {
            const long double a = (inv ? 2.0L : -2.0L) * pi * (long double)((int64_t)r * jm) /
                                  (long double)((int64_t)1 << (ls + lr));
            const long double c = cosl(a), sn = sinl(a);
            const bool f = fabsl(sn) > fabsl(c);
            const long double s = f ? sn : c;
            t[r] = f ? c / sn : sn / c;
            Sre[r] = f ? -s : s;
            Sim[r] = s;
            if (f) flags |= (int64_t)1 << (r - 1);
          }
          unsigned char* dst = base + (size_t)jm * wp_fma_rec_bytes(lr);
          auto pr = [&](double* d, long double re, long double im) {
            d[0] = (double)re;
            d[1] = (double)im;
          };
          if (lr == 3) {
            Fma8 q;
            memset(&q, 0, sizeof(q));
            for (int r = 1; r < 8; r++) q.t[r - 1] = (double)t[r];
            q.flags = flags;
            pr(q.S4, Sre[4], Sim[4]);
            pr(q.S2, Sre[2], Sim[2]);
            pr(q.R26, Sre[6] / Sre[2], Sim[6] / Sim[2]);
            pr(q.R15, Sre[5] / Sre[1], Sim[5] / Sim[1]);
            pr(q.R37, Sre[7] / Sre[3], Sim[7] / Sim[3]);
            pr(q.R13, Sre[3] / Sre[1], Sim[3] / Sim[1]);
            pr(q.M, Sre[3] / Sim[1], Sim[3] / Sre[1]);
            pr(q.S1, Sre[1], Sim[1]);
            q.h1 = (double)(Sim[1] / sqrtl(2.0L));
            q.sg1 = (double)(Sre[1] / Sim[1]);
            memcpy(dst, &q, sizeof(q));
          } else if (lr == 2) {
            Fma4 q;
            memset(&q, 0, sizeof(q));
            for (int r = 1; r < 4; r++) q.t[r - 1] = (double)t[r];
            q.flags = flags;
            pr(q.S2, Sre[2], Sim[2]);
            pr(q.S1, Sre[1], Sim[1]);
            pr(q.R13, Sre[3] / Sre[1], Sim[3] / Sim[1]);
            memcpy(dst, &q, sizeof(q));
          } else {
            Fma2 q;
            memset(&q, 0, sizeof(q));
            q.t = (double)t[1];
            q.flags = flags;
            pr(q.S, Sre[1], Sim[1]);
            memcpy(dst, &q, sizeof(q));
          }
        }
      }
      ls += lr;
    }
  }
}

}  // namespace wp
