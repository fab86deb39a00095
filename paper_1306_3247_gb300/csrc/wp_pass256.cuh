// Two-stage pass kernels for complex64 lines of 256 points (the 256^3 and 256^2 grids).
//
// One pass applies, along one axis, the operations of the split step of Sec. 2.1 that
// its flags select (inverse FFT, potential phase, forward FFT, kinetic round trip:
// eq. (splitop) with the transforms of eq. (ft)), as the Stockham kernels of
// wp_kernels.cuh do, but with a transform laid out for fewer instructions and no block
// barriers:
//
//  * A line of n = 256 = 16 x 16 points is held by 16 threads (half a warp), 16 points
//    each: thread t holds the points t + 16 r, r = 0..15 ("natural distribution").
//  * A transform is two radix-16 stages in registers (four-step form): the 16-point
//    DFT over r of each thread's points, a twiddle exp(-+2 pi i t k1/256), a transpose
//    of the 16 x 16 line through the warp's own shared memory, and the 16-point DFT
//    over t. Its output comes back in the natural distribution, so an inverse
//    transform, the potential phase and a forward transform chain in registers.
//  * Only the two threads groups of a warp share a shared-memory region: the transposes
//    synchronise the warp, never the block.
//  * Contiguous axis: the points are read and written directly (16 consecutive points
//    of a line per half warp, 128 bytes). Strided axis: a block stages 16 adjacent
//    columns (128-byte row segments, 16-byte accesses) through shared memory, with one
//    block barrier after the load and one before the store.
//
// Factors with a table (twiddles, kinetic and potential factors) are applied as one
// rounding of the exact product with the high + low FP32 parts (cmul2 / apply_factor_rec),
// which keeps the rounding unbiased: a plain FP32 factor has |w| != 1 by up to 6e-8 and
// the same factors act on the same data every step, which drifts the norm.
#pragma once

#include "wp_kernels.cuh"

namespace wp {
namespace p256 {

constexpr int kLogN = 8;
constexpr int kN = 1 << kLogN;
constexpr int kLines = 16;      // lines per block: 2 per warp
constexpr int kThreads = 256;
constexpr int kLS = 273;        // shared-memory elements per line region (16 x 17 transpose; odd stride)
#ifndef WP_P256_MIN_BLOCKS
#define WP_P256_MIN_BLOCKS 4
#endif
constexpr int kMinBlocks = WP_P256_MIN_BLOCKS;  // resident blocks per SM the register budget is set for

// exp(-2 pi i m/16), m = 1, 2: cos(pi/8), sin(pi/8), cos(pi/4) to 20 digits, split into
// the nearest float and the float nearest to the remainder.
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

// 16-point DFT in registers, natural order in: v[j] = x_j. Out: X_k in v[4 (k mod 4) + k / 4]
// (radix 4 x 4: DFTs over jb of x[ja + 4 jb], twiddles w16^(ja kb), DFTs over ja).
template <bool INV>
__device__ __forceinline__ void dft16(cx<float> (&v)[16]) {
#pragma unroll
  for (int ja = 0; ja < 4; ja++) dft4<float, INV>(v[ja], v[ja + 4], v[ja + 8], v[ja + 12]);
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
  for (int kb = 0; kb < 4; kb++) dft4<float, INV>(v[4 * kb], v[4 * kb + 1], v[4 * kb + 2], v[4 * kb + 3]);
}

__host__ __device__ constexpr int dft16_slot(int k) { return 4 * (k & 3) + (k >> 2); }

// Whole 256-point transform of the line held by a 16-thread group, natural distribution
// in and out. buf: the group's 16 x 17 transpose region; tw: the block's twiddle records,
// tw[k1 * 16 + t] = exp(-2 pi i t k1/256) as high + low parts. Synchronises the warp.
template <bool INV>
__device__ __forceinline__ void fft256(cx<float> (&v)[16], cx<float>* buf, const TwE<float>* tw, int t) {
  dft16<INV>(v);
  // v[slot(k1)] = Y[t][k1]: twiddle, then buf[k1 * 17 + t]
  __syncwarp();  // the previous transform's reads of buf are done
#pragma unroll
  for (int k1 = 0; k1 < 16; k1++) {
    cx<float> y = v[dft16_slot(k1)];
    if (k1 > 0) {
      const TwE<float> e = tw[k1 * 16 + t];
      y = INV ? cmulc2(y, e.h, e.l) : cmul2(y, e.h, e.l);
    }
    buf[k1 * 17 + t] = y;
  }
  __syncwarp();
  // thread t now plays k1 = t: v[j2] = Y[j2][t]
#pragma unroll
  for (int j2 = 0; j2 < 16; j2++) v[j2] = buf[t * 17 + j2];
  dft16<INV>(v);
  // v[slot(k2)] = X[t + 16 k2]: back to the natural distribution
  cx<float> o[16];
#pragma unroll
  for (int r = 0; r < 16; r++) o[r] = v[dft16_slot(r)];
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = o[r];
}

// Twiddle records into shared memory (all threads; the caller synchronises the block).
__device__ __forceinline__ void load_twiddles(TwE<float>* s_tw, const void* W256) {
  const float4* src = reinterpret_cast<const float4*>(W256);
  float4* dst = reinterpret_cast<float4*>(s_tw);
  for (int k = threadIdx.x; k < kN; k += blockDim.x) dst[k] = __ldg(src + k);
}

// A factor that is the product of a line factor L (the other axes) and an axis factor a
// is applied as two products, each with the exact high + low parts and one rounding:
// both roundings are unbiased, so no norm drift builds up over the steps.

// Potential phase of point i = t + 16 r of a line with record rec: additive terms (SEP)
// as the line factor and the axis records, NG Gaussian terms as exp(-i theta),
// theta = line coefficient x axis factor.
template <int NG, bool SEP>
__device__ __forceinline__ void phase256(const PassParams<float>& p, cx<float> (&v)[16], const LineRec<float>& rec,
                                         int t) {
  const float* G0 = p.G[0][p.axis];
  const float* G1 = p.G[1][p.axis];
#pragma unroll
  for (int r = 0; r < 16; r++) {
    const int i = t + 16 * r;
    cx<float> x = v[r];
    if constexpr (SEP) {
      const TwE<float> a = p.Prec[i];
      x = cmul2(cmul2(x, rec.L.h, rec.L.l), a.h, a.l);
    }
    if constexpr (NG > 0) x = apply_gauss_phase(x, rec.g[0] * __ldg(G0 + i));
    if constexpr (NG > 1) x = apply_gauss_phase(x, rec.g[1] * __ldg(G1 + i));
    v[r] = x;
  }
}

// Kinetic round trip of one line: line factor, forward FFT, axis factor, inverse FFT
// (the line factor is constant along the line, so it commutes with the transform).
__device__ __forceinline__ void kinetic256(const PassParams<float>& p, cx<float> (&v)[16], cx<float>* buf,
                                           const TwE<float>* tw, const TwE<float>& L, int t) {
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = cmul2(v[r], L.h, L.l);
  fft256<false>(v, buf, tw, t);
#pragma unroll
  for (int r = 0; r < 16; r++) {
    const TwE<float> a = p.Krec[t + 16 * r];
    v[r] = cmul2(v[r], a.h, a.l);
  }
  fft256<true>(v, buf, tw, t);
}

// Contiguous axis: tile b is lines 16 b .. 16 b + 15; warp w serves lines 16 b + 2 w + g.
// Flags: F_IFFT, F_PHASE, F_FFT (any subset, in that order). v: the thread's 16 points
// of its line, already loaded by the caller.
template <int NG, bool SEP>
__device__ __forceinline__ void contig_body(const PassParams<float>& p, int64_t tile, unsigned char* smem,
                                            cx<float> (&v)[16]) {
  TwE<float>* s_tw = reinterpret_cast<TwE<float>*>(smem);
  cx<float>* s_buf = reinterpret_cast<cx<float>*>(smem + kN * sizeof(TwE<float>));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 4, t = lane & 15;
  const int l = 2 * warp + g;
  const int64_t line = tile * kLines + l;
  cx<float>* buf = s_buf + l * kLS;
  const uint32_t f = p.flags;
  load_twiddles(s_tw, p.W256);
  __syncthreads();
  if (f & F_IFFT) fft256<true>(v, buf, s_tw, t);
  if (f & F_PHASE) {
    const LineRec<float> rec = p.lines_phase[line];
    phase256<NG, SEP>(p, v, rec, t);
  }
  if (f & F_FFT) fft256<false>(v, buf, s_tw, t);
  cx<float>* dst = p.out + (line << kLogN) + t;
#pragma unroll
  for (int r = 0; r < 16; r++) dst[16 * r] = v[r];
}

// The 16 points t + 16 r of the thread's line of a contiguous tile.
__device__ __forceinline__ void contig_load(const cx<float>* in, int64_t tile, cx<float> (&v)[16]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t line = tile * kLines + 2 * warp + (lane >> 4);
  const cx<float>* src = in + (line << kLogN) + (lane & 15);
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = src[16 * r];
}

// Strided axis (element stride 2^log_inner, log_inner >= 4): tile b is the 16 adjacent
// columns cb .. cb + 15 of outer index o. KIN: the kinetic round trip; otherwise F_FFT or
// F_IFFT. ld: the thread's 8 loads of the tile (strided_load), issued by the caller.
__device__ __forceinline__ void strided_origin(const PassParams<float>& p, int64_t tile, int64_t& o, int64_t& cb) {
  const int tpo = p.log_inner - 4;  // tiles per outer index
  o = tile >> tpo;
  cb = (tile & ((int64_t(1) << tpo) - 1)) << 4;
}

// Cooperative load: thread tau reads columns 2 c2, 2 c2 + 1 of rows tau / 8 + 32 q.
__device__ __forceinline__ void strided_load(const cx<float>* in, int log_inner, int64_t o, int64_t cb,
                                             float4 (&ld)[8]) {
  const int c2 = threadIdx.x & 7, row0 = threadIdx.x >> 3;
  const cx<float>* gin = in + (((o << kLogN) + row0) << log_inner) + cb + 2 * c2;
  const int64_t rstep = int64_t(32) << log_inner;
#pragma unroll
  for (int q = 0; q < 8; q++) ld[q] = __ldg(reinterpret_cast<const float4*>(gin + q * rstep));
}

template <bool KIN>
__device__ __forceinline__ void strided_body(const PassParams<float>& p, int64_t o, int64_t cb, unsigned char* smem,
                                             const float4 (&ld)[8]) {
  TwE<float>* s_tw = reinterpret_cast<TwE<float>*>(smem);
  cx<float>* s_tile = reinterpret_cast<cx<float>*>(smem + kN * sizeof(TwE<float>));
  const int c2 = threadIdx.x & 7, row0 = threadIdx.x >> 3;
  load_twiddles(s_tw, p.W256);
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int row = row0 + 32 * q;
    s_tile[(2 * c2) * kLS + row] = mk(ld[q].x, ld[q].y);
    s_tile[(2 * c2 + 1) * kLS + row] = mk(ld[q].z, ld[q].w);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 4, t = lane & 15;
  const int l = 2 * warp + g;
  cx<float>* reg = s_tile + l * kLS;
  cx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = reg[t + 16 * r];
  if constexpr (KIN) {
    const TwE<float> L = p.lines_kin[cb + l].L;
    kinetic256(p, v, reg, s_tw, L, t);
  } else if (p.flags & F_IFFT) {
    fft256<true>(v, reg, s_tw, t);
  } else {
    fft256<false>(v, reg, s_tw, t);
  }
  __syncwarp();  // the last transpose's reads of the region are done
#pragma unroll
  for (int r = 0; r < 16; r++) reg[t + 16 * r] = v[r];
  __syncthreads();
  cx<float>* gout = p.out + (((o << kLogN) + row0) << p.log_inner) + cb + 2 * c2;
  const int64_t rstep = int64_t(32) << p.log_inner;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int row = row0 + 32 * q;
    const cx<float> a = s_tile[(2 * c2) * kLS + row], b = s_tile[(2 * c2 + 1) * kLS + row];
    *reinterpret_cast<float4*>(gout + q * rstep) = make_float4(a.re, a.im, b.re, b.im);
  }
}

// NG Gaussian terms, SEP additive terms in the potential (one kernel per kind keeps the
// unrolled phase code small).
template <int NG, bool SEP>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_pass256_contig(const PassParams<float> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the line loads are issued before the twiddle table's (their latencies overlap)
  cx<float> v[16];
  contig_load(p.in, blockIdx.x, v);
  contig_body<NG, SEP>(p, blockIdx.x, smem_raw, v);
}

template <bool KIN>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_pass256_strided(const PassParams<float> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int64_t o, cb;
  strided_origin(p, blockIdx.x, o, cb);
  float4 ld[8];
  strided_load(p.in, p.log_inner, o, cb, ld);
  strided_body<KIN>(p, o, cb, smem_raw, ld);
}

// Batched form: block b of the launch is block block_off + b of a class-sorted block
// list (block_inst: its instance; tile_start[k]: first block of instance k). The block
// loads its tile with only the state pointer and the axis stride of its instance, then
// copies the instance's parameters to shared memory, so the two latencies overlap; the
// body is the one of the single-instance kernels, so an instance gives the same bits
// alone and in a batch.
template <bool CONTIG, bool KIN, int NG = 0, bool SEP = false>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_pass256_batch(const PassParams<float>* __restrict__ params,
                                                               const int64_t* __restrict__ tile_start,
                                                               const int* __restrict__ block_inst, int64_t block_off,
                                                               uint32_t flags, int khalf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) unsigned char raw[sizeof(PassParams<float>)];
  PassParams<float>& p = *reinterpret_cast<PassParams<float>*>(raw);
  const int64_t blk = block_off + blockIdx.x;
  const int inst = block_inst[blk];
  const int64_t tile = blk - tile_start[inst];
  const cx<float>* in = params[inst].in;
  [[maybe_unused]] cx<float> v[16];
  [[maybe_unused]] float4 ld[8];
  [[maybe_unused]] int64_t o = 0, cb = 0;
  if constexpr (CONTIG) {
    contig_load(in, tile, v);
  } else {
    const int li = params[inst].log_inner;
    const int tpo = li - 4;
    o = tile >> tpo;
    cb = (tile & ((int64_t(1) << tpo) - 1)) << 4;
    strided_load(in, li, o, cb, ld);
  }
  const int* src = reinterpret_cast<const int*>(&params[inst]);
  for (int k = threadIdx.x; k < (int)(sizeof(PassParams<float>) / sizeof(int)); k += blockDim.x)
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

// Dynamic shared memory of either kernel: the twiddle records and 16 line regions.
constexpr size_t kSmem = kN * sizeof(TwE<float>) + (size_t)kLines * kLS * sizeof(cx<float>);

}  // namespace p256
}  // namespace wp
