// Two-stage pass kernels for lines of 256 points (the 256^3 and 256^2 grids), complex64
// (T = float) and the float-float complex128-accuracy form (T = ff).
//
// One pass applies, along one axis, the operations of the split step of Sec. 2.1 that
// its flags select (inverse FFT, potential phase, forward FFT, kinetic round trip:
// eq. (splitop) with the transforms of eq. (ft)), as the Stockham kernels of
// wp_kernels.cuh do, but with a transform laid out for fewer instructions and no block
// barriers:
//
//  * A line of n = 256 = 16 x 16 points is held by 16 threads (half a warp), 16 points
//    each: thread t holds the points t + 16 r, r = 0..15 ("natural distribution"). A
//    block holds 16 lines (complex64, 256 threads) or 8 (float-float, 128 threads: its
//    16-byte points need twice the registers and shared memory).
//  * A transform is two radix-16 stages in registers (four-step form): the 16-point
//    DFT over r of each thread's points, a twiddle exp(-+2 pi i t k1/256), a transpose
//    of the 16 x 16 line through the warp's own shared memory, and the 16-point DFT
//    over t. Its output comes back in the natural distribution, so an inverse
//    transform, the potential phase and a forward transform chain in registers.
//  * Only the two threads groups of a warp share a shared-memory region: the transposes
//    synchronise the warp, never the block.
//  * Contiguous axis: the points are read and written directly (16 consecutive points
//    of a line per half warp). Strided axis: a block stages its adjacent columns
//    (128-byte row segments, 16-byte accesses) through shared memory, with one block
//    barrier after the load and one before the store.
//
// complex64: factors with a table (twiddles, kinetic and potential factors) are applied as
// one rounding of the exact product with the high + low FP32 parts (cmul2), which keeps
// the rounding unbiased: a plain FP32 factor has |w| != 1 by up to 6e-8 and the same
// factors act on the same data every step, which drifts the norm. Float-float applies
// its records with error-free products (about 48 significant bits).
#pragma once

#include "wp_kernels.cuh"

namespace wp {
namespace p256 {

constexpr int kLogN = 8;
constexpr int kN = 1 << kLogN;
constexpr int kLS = 273;  // shared-memory elements per line region (16 x 17 transpose; odd stride)

// Block shape of each form: lines per block (2 per warp) and the resident blocks per SM
// the register budget is set for (complex64: 64 registers; float-float: 128).
template <class T>
struct Shape;
template <>
struct Shape<float> {
  static constexpr int kLogLines = 4, kMinBlocks = 4;
};
template <>
struct Shape<ff> {
  static constexpr int kLogLines = 3, kMinBlocks = 4;
};
template <class T>
__host__ __device__ constexpr int lines_of() { return 1 << Shape<T>::kLogLines; }
template <class T>
__host__ __device__ constexpr int threads_of() { return 16 << Shape<T>::kLogLines; }
// Dynamic shared memory: the twiddle records and one region per line (the same for both).
template <class T>
__host__ __device__ constexpr size_t smem_of() { return kN * sizeof(TwE<T>) + (size_t)lines_of<T>() * kLS * sizeof(cx<T>); }
static_assert(smem_of<float>() == kPass256Smem && smem_of<ff>() == kPass256Smem, "host copy of the size");
constexpr size_t kSmem = kPass256Smem;

// exp(-2 pi i m/16), m = 1, 2: cos(pi/8), sin(pi/8), cos(pi/4) to 20 digits, split into
// the nearest float and the float nearest to the remainder (complex64), or held as
// float-float values.
constexpr double kC1 = 0.92387953251128675613;
constexpr double kS1 = 0.38268343236508977173;
constexpr double kC2 = 0.70710678118654752440;
constexpr float kC1h = (float)kC1, kC1l = (float)(kC1 - (double)kC1h);
constexpr float kS1h = (float)kS1, kS1l = (float)(kS1 - (double)kS1h);
constexpr float kC2h = (float)kC2, kC2l = (float)(kC2 - (double)kC2h);

// x (h + l) with one final rounding.
__device__ __forceinline__ float mulhl(float x, float h, float l) { return fmaf(x, h, x * l); }

// v (C + i S) with C = ch + cl, S = sh + sl, one final rounding per component.
__device__ __forceinline__ cx<float> cmul_hl(cx<float> v, float ch, float cl, float sh, float sl) {
  const float r = fmaf(v.re, cl, -(v.im * sl));
  const float i = fmaf(v.re, sl, v.im * cl);
  return mk(fmaf(v.re, ch, fmaf(-v.im, sh, r)), fmaf(v.re, sh, fmaf(v.im, ch, i)));
}

// v w16^m for the forward transform (w16 = exp(-2 pi i/16)), v conj(w16^m) for the inverse.
template <int M, bool INV>
__device__ __forceinline__ cx<float> w16(cx<float> v) {
  constexpr float sg = INV ? 1.0f : -1.0f;  // sign of the imaginary part of w16^1
  if constexpr (M == 1) {
    return cmul_hl(v, kC1h, kC1l, sg * kS1h, sg * kS1l);
  } else if constexpr (M == 3) {
    return cmul_hl(v, kS1h, kS1l, sg * kC1h, sg * kC1l);
  } else if constexpr (M == 9) {
    return cmul_hl(v, -kC1h, -kC1l, -sg * kS1h, -sg * kS1l);
  } else if constexpr (M == 2) {
    // (1 + sg i) / sqrt(2): ((a - sg b) + i (b + sg a)) / sqrt(2)
    const float u = INV ? v.re - v.im : v.re + v.im;
    const float w = INV ? v.im + v.re : v.im - v.re;
    return mk(mulhl(u, kC2h, kC2l), mulhl(w, kC2h, kC2l));
  } else if constexpr (M == 6) {
    // (-1 + sg i) / sqrt(2)
    const float u = INV ? -v.re - v.im : v.im - v.re;
    const float w = INV ? v.re - v.im : -v.re - v.im;
    return mk(mulhl(u, kC2h, kC2l), mulhl(w, kC2h, kC2l));
  } else {
    static_assert(M == 4, "w16 exponent");
    return rot<float, INV>(v);  // -i forward, +i inverse
  }
}
template <int M, bool INV>
__device__ __forceinline__ cx<ff> w16(cx<ff> v) {
  constexpr double sg = INV ? 1.0 : -1.0;
  if constexpr (M == 1) {
    return cmul(v, mk(ff(kC1), ff(sg * kS1)));
  } else if constexpr (M == 3) {
    return cmul(v, mk(ff(kS1), ff(sg * kC1)));
  } else if constexpr (M == 9) {
    return cmul(v, mk(ff(-kC1), ff(-sg * kS1)));
  } else if constexpr (M == 2) {
    const ff u = INV ? ff_add_raw(v.re, -v.im) : ff_add_raw(v.re, v.im);
    const ff w = INV ? ff_add_raw(v.im, v.re) : ff_add_raw(v.im, -v.re);
    return mk(mul_rsqrt2(u), mul_rsqrt2(w));
  } else if constexpr (M == 6) {
    const ff u = INV ? ff_add_raw(-v.re, -v.im) : ff_add_raw(v.im, -v.re);
    const ff w = INV ? ff_add_raw(v.re, -v.im) : ff_add_raw(-v.re, -v.im);
    return mk(mul_rsqrt2(u), mul_rsqrt2(w));
  } else {
    static_assert(M == 4, "w16 exponent");
    return rot<ff, INV>(v);
  }
}

// 16-point DFT in registers, natural order in: v[j] = x_j. Out: X_k in v[4 (k mod 4) + k / 4]
// (radix 4 x 4: DFTs over jb of x[ja + 4 jb], twiddles w16^(ja kb), DFTs over ja).
template <bool INV, class T>
__device__ __forceinline__ void dft16(cx<T> (&v)[16]) {
#pragma unroll
  for (int ja = 0; ja < 4; ja++) dft4<T, INV>(v[ja], v[ja + 4], v[ja + 8], v[ja + 12]);
  v[5] = w16<1, INV>(v[5]);
  v[9] = w16<2, INV>(v[9]);
  v[13] = w16<3, INV>(v[13]);
  v[6] = w16<2, INV>(v[6]);
  v[10] = w16<4, INV>(v[10]);
  v[14] = w16<6, INV>(v[14]);
  v[7] = w16<3, INV>(v[7]);
  v[11] = w16<6, INV>(v[11]);
  v[15] = w16<9, INV>(v[15]);
#pragma unroll
  for (int kb = 0; kb < 4; kb++) dft4<T, INV>(v[4 * kb], v[4 * kb + 1], v[4 * kb + 2], v[4 * kb + 3]);
}

__host__ __device__ constexpr int dft16_slot(int k) { return 4 * (k & 3) + (k >> 2); }

// Whole 256-point transform of the line held by a 16-thread group, natural distribution
// in and out. buf: the group's 16 x 17 transpose region; tw: the block's twiddle records,
// tw[k1 * 16 + t] = exp(-2 pi i t k1/256). Synchronises the warp.
template <bool INV, class T>
__device__ __forceinline__ void fft256(cx<T> (&v)[16], cx<T>* buf, const TwE<T>* tw, int t) {
  dft16<INV>(v);
  // v[slot(k1)] = Y[t][k1]: twiddle, then buf[k1 * 17 + t]
  __syncwarp();  // the previous transform's reads of buf are done
#pragma unroll
  for (int k1 = 0; k1 < 16; k1++) {
    cx<T> y = v[dft16_slot(k1)];
    if (k1 > 0) y = tw_apply<INV>(y, tw[k1 * 16 + t]);
    buf[k1 * 17 + t] = y;
  }
  __syncwarp();
  // thread t now plays k1 = t: v[j2] = Y[j2][t]
#pragma unroll
  for (int j2 = 0; j2 < 16; j2++) v[j2] = buf[t * 17 + j2];
  dft16<INV>(v);
  // v[slot(k2)] = X[t + 16 k2]: back to the natural distribution
  cx<T> o[16];
#pragma unroll
  for (int r = 0; r < 16; r++) o[r] = v[dft16_slot(r)];
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = o[r];
}

// Twiddle records (16 bytes each) into shared memory (all threads; the caller
// synchronises the block).
template <class T>
__device__ __forceinline__ void load_twiddles(TwE<T>* s_tw, const void* W256) {
  const float4* src = reinterpret_cast<const float4*>(W256);
  float4* dst = reinterpret_cast<float4*>(s_tw);
  for (int k = threadIdx.x; k < kN; k += blockDim.x) dst[k] = __ldg(src + k);
}

// Axis table entries of the Gaussian terms.
__device__ __forceinline__ float table_value(const float* p) { return __ldg(p); }
__device__ __forceinline__ ff table_value(const ff* p) { return *p; }

// Gaussian terms skip whole lines whose coefficient is negligible (gauss_line_active).

// A factor that is the product of a line factor L (the other axes) and an axis factor a:
// complex64 forms the product a L exactly (error-free products and sums of the high + low
// parts) and rounds v a L once. Two roundings (v L, then (v L) a) drift the norm of a
// nearly periodic state by about 1e-8 per step: its points repeat, and so do their
// rounding errors (measured: 1.3e-5 after 1000 steps of the 128^2 trapped packet, against
// 1e-6 with one rounding). Float-float applies the two records one after the other
// (error-free complex products, about 48 bits).
__device__ __forceinline__ cx<float> mul_line_axis(cx<float> v, const TwE<float>& L, const TwE<float>& a) {
  return apply_factor(v, a.h, a.l, L.h, L.l);
}
__device__ __forceinline__ cx<ff> mul_line_axis(cx<ff> v, const TwE<ff>& L, const TwE<ff>& a) {
  return tw_apply<false>(tw_apply<false>(v, L), a);
}

// Potential phase of point i = t + 16 r of a line with record rec: additive terms (SEP)
// as the line factor and the axis records, NG Gaussian terms as exp(-i theta),
// theta = line coefficient x axis factor.
template <int NG, bool SEP, class T>
__device__ __forceinline__ void phase256(const PassParams<T>& p, cx<T> (&v)[16], const LineRec<T>& rec, int t) {
  const T* G0 = p.G[0][p.axis];
  const T* G1 = p.G[1][p.axis];
  const bool g0 = NG > 0 && gauss_line_active(rec.g[0]);
  const bool g1 = NG > 1 && gauss_line_active(rec.g[1]);
#pragma unroll
  for (int r = 0; r < 16; r++) {
    const int i = t + 16 * r;
    cx<T> x = v[r];
    if constexpr (SEP) x = mul_line_axis(x, rec.L, p.Prec[i]);
    if constexpr (NG > 0)
      if (g0) x = apply_gauss_phase(x, rec.g[0] * table_value(G0 + i));
    if constexpr (NG > 1)
      if (g1) x = apply_gauss_phase(x, rec.g[1] * table_value(G1 + i));
    v[r] = x;
  }
}

// Kinetic round trip of one line: forward FFT, kinetic factor (line x axis), inverse FFT.
template <class T>
__device__ __forceinline__ void kinetic256(const PassParams<T>& p, cx<T> (&v)[16], cx<T>* buf, const TwE<T>* tw,
                                           const TwE<T>& L, int t) {
  fft256<false>(v, buf, tw, t);
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = mul_line_axis(v[r], L, p.Krec[t + 16 * r]);
  fft256<true>(v, buf, tw, t);
}

// Observable sums of a two-stage pass (complex64; the tables and the per-line rows of the
// Stockham kernels' sums). Position sums of the thread's 16 points (after the potential
// phase): |psi|^2 times 1, x, x^2, the additive potential, the Gaussian axis factors,
// and conj(psi0) psi (psi0: the thread's first point of the initial state).
template <class T>
__device__ __forceinline__ void pos_sums256(const PassParams<T>& p, const cx<T> (&v)[16], const cx<T>* psi0, int t,
                                            T (&q)[8]) {
  const T* G0 = p.G[0][p.axis];
  const T* G1 = p.G[1][p.axis];
  const bool ac = (p.flags & F_AUTOCORR) != 0;
#pragma unroll
  for (int r = 0; r < 16; r++) {
    const int i = t + 16 * r;
    const T rho = norm2(v[r]);
    const cx<T> xx = p.Ox[i];
    q[0] = q[0] + rho;
    q[1] = madd(xx.re, rho, q[1]);
    q[2] = madd(xx.im, rho, q[2]);
    q[3] = madd(p.AT[i], rho, q[3]);
    if (p.ngauss > 0) q[4] = madd(G0[i], rho, q[4]);
    if (p.ngauss > 1) q[5] = madd(G1[i], rho, q[5]);
    if (ac) {
      const cx<T> c = cmulc(v[r], psi0[16 * r]);
      q[6] = q[6] + c.re;
      q[7] = q[7] + c.im;
    }
  }
}

// Momentum sums of the thread's 16 points after the forward transform: |psi_hat|^2 times
// 1, k, k^2.
template <class T>
__device__ __forceinline__ void mom_sums256(const PassParams<T>& p, const cx<T> (&v)[16], int t, T (&q)[8]) {
#pragma unroll
  for (int r = 0; r < 16; r++) {
    const T rho = norm2(v[r]);
    const cx<T> kk = p.Ok[t + 16 * r];
    q[0] = q[0] + rho;
    q[1] = madd(kk.re, rho, q[1]);
    q[2] = madd(kk.im, rho, q[2]);
  }
}

// The block's partial row. The 16 threads of a line combine their sums by xor
// butterflies (every lane then holds the line sums) and lane t forms slot t of the line's
// row (the quantities obs_line_row forms in FP64 for the Stockham kernels), in FP32 and
// scaled so that no product leaves the FP32 range in any units: slot t holds its value
// divided by a power of two s_t that is the same for every line (oscale_x[d] or its
// square for the position moments of axis d, oscale_k[d] for the momentum of axis d,
// k2s for |k|^2). The block's lines are then summed in order in FP64 and multiplied by
// s_t (exactly) into partials[blockIdx.x]. The row is formed in FP32 because GB300 runs
// FP64 at 1/64 of the FP32 rate: an FP64 row, one branch per slot, made the observable
// passes 25-70 us longer than the plain ones on the 256^3 grid. o, c: the line's outer
// index and column, as grid_index takes them. Every thread of the block calls it.
template <class T>
__device__ __forceinline__ void obs256_partials(const PassParams<T>& p, T (&q)[8], int64_t o, int64_t c, int l,
                                                int t) {
  static_assert(std::is_same<T, float>::value, "the two-stage kernels form sums in complex64 only");
  static_assert(NQ == 16, "one row slot per lane of a line");
  __shared__ float red[lines_of<T>()][NQ];
#pragma unroll
  for (int s = 8; s > 0; s >>= 1)
#pragma unroll
    for (int j = 0; j < 8; j++) q[j] = q[j] + shfl_xor(q[j], s);
  const Geom& g = p.g;
  const int ax = p.axis, nd = g.ndim;
  const bool pos = (p.flags & F_OBS_POS) != 0;
  int gi[3];
  grid_index(g, ax, o, c, 0, gi);
  const float lt0 = q[0];
  float v = 0.0f;
  if (pos) {
    // slots Q_X + d and Q_XX + d
    const bool sq = t >= Q_XX && t < Q_XX + 3;
    const int d = sq ? t - Q_XX : (t >= Q_X && t < Q_X + 3 ? t - Q_X : 0);
    const int gd = d == 0 ? gi[0] : (d == 1 ? gi[1] : gi[2]);
    const float xr = fmaf((float)gd, d == 0 ? g.dxr[0] : (d == 1 ? g.dxr[1] : g.dxr[2]),
                          d == 0 ? g.xr0[0] : (d == 1 ? g.xr0[1] : g.xr0[2]));
    const float mom = d == ax ? (sq ? q[2] : q[1]) : (sq ? xr * xr : xr) * lt0;
    // the line's potential parts on the other axes
    float A = 0.0f, P0 = 0.0f, P1 = 0.0f;
#pragma unroll
    for (int e = 0; e < 3; e++)
      if (e < nd && e != ax) A += p.ATax[e][gi[e]];
    if (p.ngauss > 0) {
      P0 = (float)p.ctrl->gcoef[0];
#pragma unroll
      for (int e = 0; e < 3; e++)
        if (e < nd && e != ax) P0 *= p.G[0][e][gi[e]];
    }
    if (p.ngauss > 1) {
      P1 = (float)p.ctrl->gcoef[1];
#pragma unroll
      for (int e = 0; e < 3; e++)
        if (e < nd && e != ax) P1 *= p.G[1][e][gi[e]];
    }
    if (t == Q_RHO)
      v = lt0;
    else if (t < Q_V)
      v = d < nd ? mom : 0.0f;
    else if (t == Q_V)
      v = fmaf(P1, q[5], fmaf(P0, q[4], fmaf(A, lt0, q[3])));
    else if (t == Q_AC_RE)
      v = q[6];
    else if (t == Q_AC_IM)
      v = q[7];
  } else {
    // k_e / oscale_k[e] of the line on the other axes
    float kr[3];
#pragma unroll
    for (int e = 0; e < 3; e++) {
      const int n = 1 << g.ln[e];
      kr[e] = (float)(gi[e] < (n >> 1) ? gi[e] : gi[e] - n) * g.kr[e];
    }
    if (t == Q_RHOK) {
      v = lt0;
    } else if (t >= Q_K && t < Q_K + 3) {
      const int d = t - Q_K;
      v = d >= nd ? 0.0f : (d == ax ? q[1] : (d == 0 ? kr[0] : (d == 1 ? kr[1] : kr[2])) * lt0);
    } else if (t == Q_K2) {
      float k2 = 0.0f;
#pragma unroll
      for (int e = 0; e < 3; e++)
        if (e < nd && e != ax) k2 = fmaf(kr[e] * kr[e], g.k2r[e], k2);
      v = fmaf(q[2], ax == 0 ? g.k2r[0] : (ax == 1 ? g.k2r[1] : g.k2r[2]), k2 * lt0);
    }
  }
  red[l][t] = v;
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int s = threadIdx.x;
    double sum = 0.0;
    for (int k = 0; k < lines_of<T>(); k++) sum += (double)red[k][s];
    double scale = 1.0;
    if (pos) {
      if (s >= Q_X && s < Q_X + 3) scale = g.oscale_x[s - Q_X];
      if (s >= Q_XX && s < Q_XX + 3) scale = g.oscale_x[s - Q_XX] * g.oscale_x[s - Q_XX];
    } else {
      if (s >= Q_K && s < Q_K + 3) scale = g.oscale_k[s - Q_K];
      if (s == Q_K2) scale = g.k2s;
    }
    p.partials[blockIdx.x * (int64_t)NQ + s] = sum * scale;
  }
}

// Contiguous axis: tile b is lines L b .. L b + L - 1 (L lines per block); warp w serves
// lines L b + 2 w + g. Flags: F_IFFT, F_PHASE, F_FFT (any subset, in that order); with
// OBS also F_OBS_POS (position sums after the phase, before the forward transform),
// F_AUTOCORR and F_NO_STORE. v: the thread's 16 points of its line, already loaded by the
// caller.
template <int NG, bool SEP, bool OBS = false, class T>
__device__ __forceinline__ void contig_body(const PassParams<T>& p, int64_t tile, unsigned char* smem,
                                            cx<T> (&v)[16]) {
  TwE<T>* s_tw = reinterpret_cast<TwE<T>*>(smem);
  cx<T>* s_buf = reinterpret_cast<cx<T>*>(smem + kN * sizeof(TwE<T>));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 4, t = lane & 15;
  const int l = 2 * warp + g;
  const int64_t line = tile * lines_of<T>() + l;
  cx<T>* buf = s_buf + l * kLS;
  const uint32_t f = p.flags;
  load_twiddles(s_tw, p.W256);
  __syncthreads();
  if (f & F_IFFT) fft256<true>(v, buf, s_tw, t);
  if (f & F_PHASE) {
    const LineRec<T> rec = p.lines_phase[line];
    phase256<NG, SEP>(p, v, rec, t);
  }
  [[maybe_unused]] T q[8];
  if constexpr (OBS) {
#pragma unroll
    for (int j = 0; j < 8; j++) q[j] = T(0);
    if (f & F_OBS_POS) pos_sums256(p, v, p.psi0 + (line << kLogN) + t, t, q);
  }
  if (f & F_FFT) fft256<false>(v, buf, s_tw, t);
  if (!(OBS && (f & F_NO_STORE))) {
    cx<T>* dst = p.out + (line << kLogN) + t;
#pragma unroll
    for (int r = 0; r < 16; r++) dst[16 * r] = v[r];
  }
  if constexpr (OBS) obs256_partials(p, q, line, 0, l, t);
}

// The 16 points t + 16 r of the thread's line of a contiguous tile.
template <class T>
__device__ __forceinline__ void contig_load(const cx<T>* in, int64_t tile, cx<T> (&v)[16]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t line = tile * lines_of<T>() + 2 * warp + (lane >> 4);
  const cx<T>* src = in + (line << kLogN) + (lane & 15);
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = src[16 * r];
}

// Strided axis (element stride 2^log_inner, log_inner >= log2 L): tile b is the L
// adjacent columns cb .. cb + L - 1 of outer index o. The tile is moved in 16-byte
// vectors of E = 16 / sizeof(cx<T>) points: 8 vectors per row (128 bytes), rows tau / 8 +
// (threads / 8) q for thread tau, Q = 256 / (threads / 8) of them per thread.
template <class T>
struct Stage {
  static constexpr int E = 16 / (int)sizeof(cx<T>);
  static constexpr int RP = threads_of<T>() / 8;  // rows per round
  static constexpr int Q = kN / RP;               // rounds
};

template <class T>
__device__ __forceinline__ void strided_origin(int log_inner, int64_t tile, int64_t& o, int64_t& cb) {
  const int tpo = log_inner - Shape<T>::kLogLines;  // tiles per outer index
  o = tile >> tpo;
  cb = (tile & ((int64_t(1) << tpo) - 1)) << Shape<T>::kLogLines;
}

template <class T>
__device__ __forceinline__ void strided_load(const cx<T>* in, int log_inner, int64_t o, int64_t cb,
                                             float4 (&ld)[Stage<T>::Q]) {
  const int c2 = threadIdx.x & 7, row0 = threadIdx.x >> 3;
  const cx<T>* gin = in + (((o << kLogN) + row0) << log_inner) + cb + Stage<T>::E * c2;
  const int64_t rstep = int64_t(Stage<T>::RP) << log_inner;
#pragma unroll
  for (int q = 0; q < Stage<T>::Q; q++) ld[q] = __ldg(reinterpret_cast<const float4*>(gin + q * rstep));
}

// OBS (complex64, forward transform only): the momentum sums after the transform, and
// F_NO_STORE.
template <bool KIN, bool OBS = false, class T>
__device__ __forceinline__ void strided_body(const PassParams<T>& p, int64_t o, int64_t cb, unsigned char* smem,
                                             const float4 (&ld)[Stage<T>::Q]) {
  using S = Stage<T>;
  TwE<T>* s_tw = reinterpret_cast<TwE<T>*>(smem);
  cx<T>* s_tile = reinterpret_cast<cx<T>*>(smem + kN * sizeof(TwE<T>));
  const int c2 = threadIdx.x & 7, row0 = threadIdx.x >> 3;
  load_twiddles(s_tw, p.W256);
#pragma unroll
  for (int q = 0; q < S::Q; q++) {
    const int row = row0 + S::RP * q;
    if constexpr (S::E == 2) {
      s_tile[(2 * c2) * kLS + row] = mk(ld[q].x, ld[q].y);
      s_tile[(2 * c2 + 1) * kLS + row] = mk(ld[q].z, ld[q].w);
    } else {
      *reinterpret_cast<float4*>(&s_tile[c2 * kLS + row]) = ld[q];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 4, t = lane & 15;
  const int l = 2 * warp + g;
  cx<T>* reg = s_tile + l * kLS;
  cx<T> v[16];
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = reg[t + 16 * r];
  if constexpr (KIN) {
    const TwE<T> L = p.lines_kin[cb + l].L;
    kinetic256(p, v, reg, s_tw, L, t);
  } else if (p.flags & F_IFFT) {
    fft256<true>(v, reg, s_tw, t);
  } else {
    fft256<false>(v, reg, s_tw, t);
  }
  [[maybe_unused]] T qs[8];
  if constexpr (OBS) {
#pragma unroll
    for (int j = 0; j < 8; j++) qs[j] = T(0);
    mom_sums256(p, v, t, qs);
    if (p.flags & F_NO_STORE) {
      obs256_partials(p, qs, o, cb + l, l, t);
      return;
    }
  }
  __syncwarp();  // the last transpose's reads of the region are done
#pragma unroll
  for (int r = 0; r < 16; r++) reg[t + 16 * r] = v[r];
  __syncthreads();
  cx<T>* gout = p.out + (((o << kLogN) + row0) << p.log_inner) + cb + S::E * c2;
  const int64_t rstep = int64_t(S::RP) << p.log_inner;
#pragma unroll
  for (int q = 0; q < S::Q; q++) {
    const int row = row0 + S::RP * q;
    float4 w;
    if constexpr (S::E == 2) {
      const cx<float> a = s_tile[(2 * c2) * kLS + row], b = s_tile[(2 * c2 + 1) * kLS + row];
      w = make_float4(a.re, a.im, b.re, b.im);
    } else {
      w = *reinterpret_cast<const float4*>(&s_tile[c2 * kLS + row]);
    }
    *reinterpret_cast<float4*>(gout + q * rstep) = w;
  }
  if constexpr (OBS) obs256_partials(p, qs, o, cb + l, l, t);
}

// NG Gaussian terms, SEP additive terms in the potential (one kernel per kind keeps the
// unrolled phase code small).
// OBS: the variant with the position sums (complex64).
template <class T, int NG, bool SEP, bool OBS = false>
__global__ void __launch_bounds__(threads_of<T>(), Shape<T>::kMinBlocks) k_pass256_contig(const PassParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the line loads are issued before the twiddle table's (their latencies overlap)
  cx<T> v[16];
  contig_load(p.in, blockIdx.x, v);
  contig_body<NG, SEP, OBS>(p, blockIdx.x, smem_raw, v);
}

template <class T, bool KIN, bool OBS = false>
__global__ void __launch_bounds__(threads_of<T>(), Shape<T>::kMinBlocks) k_pass256_strided(const PassParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int64_t o, cb;
  strided_origin<T>(p.log_inner, blockIdx.x, o, cb);
  float4 ld[Stage<T>::Q];
  strided_load(p.in, p.log_inner, o, cb, ld);
  strided_body<KIN, OBS>(p, o, cb, smem_raw, ld);
}

// Batched form: block-list entry blk is tile blk - tile_start[inst] of instance
// inst = block_inst[blk]. The block loads its tile with only the state pointer and the
// axis stride of its instance, then copies the instance's parameters to shared memory
// (raw: a 16-byte aligned buffer of sizeof(PassParams<T>) bytes), so the two latencies
// overlap; the body is the one of the single-instance kernels, so an instance gives the
// same bits alone and in a batch.
template <class T, bool CONTIG, bool KIN, int NG = 0, bool SEP = false>
__device__ __forceinline__ void pass256_batch_body(const PassParams<T>* __restrict__ params,
                                                   const int64_t* __restrict__ tile_start,
                                                   const int* __restrict__ block_inst, int64_t blk, uint32_t flags,
                                                   int khalf, unsigned char* raw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassParams<T>& p = *reinterpret_cast<PassParams<T>*>(raw);
  const int inst = block_inst[blk];
  const int64_t tile = blk - tile_start[inst];
  const cx<T>* in = params[inst].in;
  [[maybe_unused]] cx<T> v[16];
  [[maybe_unused]] float4 ld[Stage<T>::Q];
  [[maybe_unused]] int64_t o = 0, cb = 0;
  if constexpr (CONTIG) {
    contig_load(in, tile, v);
  } else {
    const int li = params[inst].log_inner;
    strided_origin<T>(li, tile, o, cb);
    strided_load(in, li, o, cb, ld);
  }
  const int* src = reinterpret_cast<const int*>(&params[inst]);
  for (int k = threadIdx.x; k < (int)(sizeof(PassParams<T>) / sizeof(int)); k += blockDim.x)
    reinterpret_cast<int*>(raw)[k] = src[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    p.flags = flags;
    if (khalf) {
      p.Krec = p.Krec_half;
      p.lines_kin = p.lines_kin_half;
    }
  }
  __syncthreads();
  if constexpr (CONTIG)
    contig_body<NG, SEP>(p, tile, smem_raw, v);
  else
    strided_body<KIN>(p, o, cb, smem_raw, ld);
}

template <class T, bool CONTIG, bool KIN, int NG = 0, bool SEP = false>
__global__ void __launch_bounds__(threads_of<T>(), Shape<T>::kMinBlocks)
    k_pass256_batch(const PassParams<T>* __restrict__ params, const int64_t* __restrict__ tile_start,
                    const int* __restrict__ block_inst, int64_t block_off, uint32_t flags, int khalf) {
  __shared__ __align__(16) unsigned char raw[sizeof(PassParams<T>)];
  pass256_batch_body<T, CONTIG, KIN, NG, SEP>(params, tile_start, block_inst, block_off + blockIdx.x, flags, khalf,
                                              raw);
}

}  // namespace p256
}  // namespace wp
