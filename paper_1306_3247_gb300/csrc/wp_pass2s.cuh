// Two-stage pass kernels for complex64 lines of 64 and 128 points (the short axes of uneven
// 2-D batches), the companions of the 256-point kernels of wp_pass256.cuh.
//
// A line of n = 8 T points is held by T threads (T = 8 for n = 64, 16 for n = 128), 8
// points each: thread t holds the points t + T r, r = 0..7 (the natural distribution).
// A transform of the split step of Sec. 2.1 (eq. (ft)) is, in four-step form:
//   stage A: the 8-point DFT over r of each thread's points, Y[t][k1];
//   twiddle: Y[t][k1] exp(-+2 pi i t k1 / n);
//   transpose through the line's shared-memory region (the warp synchronises, never the
//   block);
//   stage B: the T-point DFT over t of each column k1. For T = 8 thread k1 takes the 8
//   values of its column and transforms them. For T = 16 (n = 128) the 16-point DFT is
//   split by a radix-2 step in frequency: thread k1 + 8 h (h = 0, 1) forms
//   z[j] = Y[j][k1] + Y[j + 8][k1] (h = 0) or (Y[j][k1] - Y[j + 8][k1]) exp(-+2 pi i j/16)
//   (h = 1), j = 0..7, and its 8-point DFT gives the outputs k2 = 2m + h.
// Either way thread t ends with X[t + T m], m = 0..7: the natural distribution again, so
// an inverse transform, the potential phase and a forward transform chain in registers.
// Factors are applied as in the 256-point kernels: records with high + low FP32 parts,
// one rounding of the exact product of a line factor and an axis factor.
#pragma once

#include "wp_pass256.cuh"

namespace wp {
namespace p2s {

constexpr int kR = 8;  // points per thread

// Blocks of 256 threads: 32 lines of 64 points or 16 lines of 128.
template <int LOGT>
struct Geo {
  static constexpr int T = 1 << LOGT;  // threads per line
  static constexpr int LOGN = LOGT + 3;
  static constexpr int N = 1 << LOGN;
  static constexpr int LOGLINES = 8 - LOGT;
  static constexpr int LINES = 1 << LOGLINES;
  static constexpr int THREADS = 256;
  // line region: the natural line (N points) and the 8 x (T + 1) transpose, odd size
  static constexpr int LS = ((N > kR * (T + 1) ? N : kR * (T + 1)) | 1);
  // twiddle records: stage twiddles [k1][t] (8 T of them), then the fold twiddles
  // exp(-2 pi i j / 16), j = 0..7 (n = 128)
  static constexpr int NTW = kR * T + (T == 16 ? 8 : 0);
  static constexpr size_t SMEM = (size_t)NTW * sizeof(TwE<float>) + (size_t)LINES * LS * sizeof(cx<float>);
};

// 8-point DFT in registers, natural order in: v[j] = x_j. Out: X_k in v[2 (k mod 4) + k / 4]
// (radix 2 x 4: DFTs over jb of x[ja + 2 jb], twiddles w8^(ja kb), DFTs over ja).
template <bool INV>
__device__ __forceinline__ void dft8(cx<float> (&v)[8]) {
  dft4<float, INV>(v[0], v[2], v[4], v[6]);
  dft4<float, INV>(v[1], v[3], v[5], v[7]);
  v[3] = p256::w16<2, INV>(v[3]);  // w8^1 = w16^2
  v[5] = rot<float, INV>(v[5]);    // w8^2
  v[7] = p256::w16<6, INV>(v[7]);  // w8^3 = w16^6
#pragma unroll
  for (int kb = 0; kb < 4; kb++) {
    const cx<float> a = v[2 * kb], b = v[2 * kb + 1];
    v[2 * kb] = cadd(a, b);
    v[2 * kb + 1] = csub(a, b);
  }
}
__host__ __device__ constexpr int dft8_slot(int k) { return 2 * (k & 3) + (k >> 2); }

// Whole transform of the line held by the thread's group; buf: its line region; tw: the
// block's twiddle records (Geo::NTW). Synchronises the warp.
template <int LOGT, bool INV>
__device__ __forceinline__ void fft(cx<float> (&v)[8], cx<float>* buf, const TwE<float>* tw, int t) {
  using G = Geo<LOGT>;
  constexpr int T = G::T;
  dft8<INV>(v);
  __syncwarp();  // the previous transform's reads of buf are done
#pragma unroll
  for (int k1 = 0; k1 < kR; k1++) {
    cx<float> y = v[dft8_slot(k1)];
    if (k1 > 0) y = tw_apply<INV>(y, tw[k1 * T + t]);
    buf[k1 * (T + 1) + t] = y;
  }
  __syncwarp();
  if constexpr (T == 8) {
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = buf[t * (T + 1) + j];
  } else {
    const int k1 = t & 7, h = t >> 3;
    const cx<float>* row = buf + k1 * (T + 1);
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const cx<float> a = row[j], b = row[j + 8];
      if (h == 0) {
        v[j] = cadd(a, b);
      } else {
        const cx<float> d = csub(a, b);
        v[j] = j == 0 ? d : tw_apply<INV>(d, tw[kR * T + j]);
      }
    }
  }
  dft8<INV>(v);
  cx<float> o[8];
#pragma unroll
  for (int m = 0; m < 8; m++) o[m] = v[dft8_slot(m)];
#pragma unroll
  for (int m = 0; m < 8; m++) v[m] = o[m];
}

template <int LOGT>
__device__ __forceinline__ void load_twiddles(TwE<float>* s_tw, const void* W) {
  const float4* src = reinterpret_cast<const float4*>(W);
  float4* dst = reinterpret_cast<float4*>(s_tw);
  for (int k = threadIdx.x; k < Geo<LOGT>::NTW; k += blockDim.x) dst[k] = __ldg(src + k);
}

// Potential phase of point i = t + T r (as phase256).
template <int LOGT, int NG, bool SEP>
__device__ __forceinline__ void phase(const PassParams<float>& p, cx<float> (&v)[8], const LineRec<float>& rec, int t) {
  const float* G0 = p.G[0][p.axis];
  const float* G1 = p.G[1][p.axis];
  const bool g0 = NG > 0 && gauss_line_active(rec.g[0]);
  const bool g1 = NG > 1 && gauss_line_active(rec.g[1]);
#pragma unroll
  for (int r = 0; r < 8; r++) {
    const int i = t + (r << LOGT);
    cx<float> x = v[r];
    if constexpr (SEP) x = p256::mul_line_axis(x, rec.L, p.Prec[i]);
    if constexpr (NG > 0)
      if (g0) x = apply_gauss_phase(x, rec.g[0] * __ldg(G0 + i));
    if constexpr (NG > 1)
      if (g1) x = apply_gauss_phase(x, rec.g[1] * __ldg(G1 + i));
    v[r] = x;
  }
}

template <int LOGT>
__device__ __forceinline__ void kinetic(const PassParams<float>& p, cx<float> (&v)[8], cx<float>* buf,
                                        const TwE<float>* tw, const TwE<float>& L, int t) {
  fft<LOGT, false>(v, buf, tw, t);
#pragma unroll
  for (int r = 0; r < 8; r++) v[r] = p256::mul_line_axis(v[r], L, p.Krec[t + (r << LOGT)]);
  fft<LOGT, true>(v, buf, tw, t);
}

// Line l of a block and thread t of its line: lines are groups of T consecutive threads.
template <int LOGT>
__device__ __forceinline__ void line_of(int& l, int& t) {
  l = threadIdx.x >> LOGT;
  t = threadIdx.x & ((1 << LOGT) - 1);
}

// Contiguous axis: tile b is lines LINES b .. LINES (b + 1) - 1. Flags: F_IFFT, F_PHASE, F_FFT.
template <int LOGT>
__device__ __forceinline__ void contig_load(const cx<float>* in, int64_t tile, cx<float> (&v)[8]) {
  int l, t;
  line_of<LOGT>(l, t);
  const cx<float>* src = in + ((tile * Geo<LOGT>::LINES + l) << Geo<LOGT>::LOGN) + t;
#pragma unroll
  for (int r = 0; r < 8; r++) v[r] = src[r << LOGT];
}

template <int LOGT, int NG, bool SEP>
__device__ __forceinline__ void contig_body(const PassParams<float>& p, int64_t tile, unsigned char* smem,
                                            cx<float> (&v)[8]) {
  using G = Geo<LOGT>;
  TwE<float>* s_tw = reinterpret_cast<TwE<float>*>(smem);
  cx<float>* s_buf = reinterpret_cast<cx<float>*>(smem + G::NTW * sizeof(TwE<float>));
  int l, t;
  line_of<LOGT>(l, t);
  const int64_t line = tile * G::LINES + l;
  cx<float>* buf = s_buf + l * G::LS;
  const uint32_t f = p.flags;
  load_twiddles<LOGT>(s_tw, p.W2s);
  __syncthreads();
  if (f & F_IFFT) fft<LOGT, true>(v, buf, s_tw, t);
  if (f & F_PHASE) {
    const LineRec<float> rec = p.lines_phase[line];
    phase<LOGT, NG, SEP>(p, v, rec, t);
  }
  if (f & F_FFT) fft<LOGT, false>(v, buf, s_tw, t);
  cx<float>* dst = p.out + (line << G::LOGN) + t;
#pragma unroll
  for (int r = 0; r < 8; r++) dst[r << LOGT] = v[r];
}

// Strided axis (log_inner >= LOGLINES): tile b is the LINES adjacent columns
// cb .. cb + LINES - 1 of outer index o, moved in 16-byte vectors (two points): VPR =
// LINES / 2 per row (128 or 256 bytes), rows tau / VPR + (THREADS / VPR) q.
template <int LOGT>
struct Stage {
  static constexpr int VPR = Geo<LOGT>::LINES / 2;   // vectors per row
  static constexpr int RP = Geo<LOGT>::THREADS / VPR;  // rows per round
  static constexpr int Q = Geo<LOGT>::N / RP;          // rounds
};

template <int LOGT>
__device__ __forceinline__ void strided_origin(int log_inner, int64_t tile, int64_t& o, int64_t& cb) {
  const int tpo = log_inner - Geo<LOGT>::LOGLINES;
  o = tile >> tpo;
  cb = (tile & ((int64_t(1) << tpo) - 1)) << Geo<LOGT>::LOGLINES;
}

template <int LOGT>
__device__ __forceinline__ void strided_load(const cx<float>* in, int log_inner, int64_t o, int64_t cb,
                                             float4 (&ld)[Stage<LOGT>::Q]) {
  const int c2 = threadIdx.x % Stage<LOGT>::VPR, row0 = threadIdx.x / Stage<LOGT>::VPR;
  const cx<float>* gin = in + (((o << Geo<LOGT>::LOGN) + row0) << log_inner) + cb + 2 * c2;
  const int64_t rstep = int64_t(Stage<LOGT>::RP) << log_inner;
#pragma unroll
  for (int q = 0; q < Stage<LOGT>::Q; q++) ld[q] = __ldg(reinterpret_cast<const float4*>(gin + q * rstep));
}

template <int LOGT, bool KIN>
__device__ __forceinline__ void strided_body(const PassParams<float>& p, int64_t o, int64_t cb, unsigned char* smem,
                                             const float4 (&ld)[Stage<LOGT>::Q]) {
  using G = Geo<LOGT>;
  using S = Stage<LOGT>;
  TwE<float>* s_tw = reinterpret_cast<TwE<float>*>(smem);
  cx<float>* s_tile = reinterpret_cast<cx<float>*>(smem + G::NTW * sizeof(TwE<float>));
  const int c2 = threadIdx.x % S::VPR, row0 = threadIdx.x / S::VPR;
  load_twiddles<LOGT>(s_tw, p.W2s);
#pragma unroll
  for (int q = 0; q < S::Q; q++) {
    const int row = row0 + S::RP * q;
    s_tile[(2 * c2) * G::LS + row] = mk(ld[q].x, ld[q].y);
    s_tile[(2 * c2 + 1) * G::LS + row] = mk(ld[q].z, ld[q].w);
  }
  __syncthreads();
  int l, t;
  line_of<LOGT>(l, t);
  cx<float>* reg = s_tile + l * G::LS;
  cx<float> v[8];
#pragma unroll
  for (int r = 0; r < 8; r++) v[r] = reg[t + (r << LOGT)];
  if constexpr (KIN) {
    const TwE<float> L = p.lines_kin[cb + l].L;
    kinetic<LOGT>(p, v, reg, s_tw, L, t);
  } else if (p.flags & F_IFFT) {
    fft<LOGT, true>(v, reg, s_tw, t);
  } else {
    fft<LOGT, false>(v, reg, s_tw, t);
  }
  __syncwarp();  // the last transpose's reads of the region are done
#pragma unroll
  for (int r = 0; r < 8; r++) reg[t + (r << LOGT)] = v[r];
  __syncthreads();
  cx<float>* gout = p.out + (((o << G::LOGN) + row0) << p.log_inner) + cb + 2 * c2;
  const int64_t rstep = int64_t(S::RP) << p.log_inner;
#pragma unroll
  for (int q = 0; q < S::Q; q++) {
    const int row = row0 + S::RP * q;
    const cx<float> a = s_tile[(2 * c2) * G::LS + row], b = s_tile[(2 * c2 + 1) * G::LS + row];
    *reinterpret_cast<float4*>(gout + q * rstep) = make_float4(a.re, a.im, b.re, b.im);
  }
}

// Resident blocks per SM the register budget is set for (8 points per thread: few
// registers).
template <int LOGT>
constexpr int min_blocks() { return 5; }

template <int LOGT, int NG, bool SEP>
__global__ void __launch_bounds__(Geo<LOGT>::THREADS, min_blocks<LOGT>()) k_pass2s_contig(const PassParams<float> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float> v[8];
  contig_load<LOGT>(p.in, blockIdx.x, v);
  contig_body<LOGT, NG, SEP>(p, blockIdx.x, smem_raw, v);
}

template <int LOGT, bool KIN>
__global__ void __launch_bounds__(Geo<LOGT>::THREADS, min_blocks<LOGT>()) k_pass2s_strided(const PassParams<float> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int64_t o, cb;
  strided_origin<LOGT>(p.log_inner, blockIdx.x, o, cb);
  float4 ld[Stage<LOGT>::Q];
  strided_load<LOGT>(p.in, p.log_inner, o, cb, ld);
  strided_body<LOGT, KIN>(p, o, cb, smem_raw, ld);
}

// Batched form (as pass256_batch_body): tile loads first, then the instance's parameters.
template <int LOGT, bool CONTIG, bool KIN, int NG = 0, bool SEP = false>
__device__ __forceinline__ void batch_body(const PassParams<float>* __restrict__ params,
                                           const int64_t* __restrict__ tile_start,
                                           const int* __restrict__ block_inst, int64_t blk, uint32_t flags, int khalf,
                                           unsigned char* raw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassParams<float>& p = *reinterpret_cast<PassParams<float>*>(raw);
  const int inst = block_inst[blk];
  const int64_t tile = blk - tile_start[inst];
  const cx<float>* in = params[inst].in;
  [[maybe_unused]] cx<float> v[8];
  [[maybe_unused]] float4 ld[Stage<LOGT>::Q];
  [[maybe_unused]] int64_t o = 0, cb = 0;
  if constexpr (CONTIG) {
    contig_load<LOGT>(in, tile, v);
  } else {
    const int li = params[inst].log_inner;
    strided_origin<LOGT>(li, tile, o, cb);
    strided_load<LOGT>(in, li, o, cb, ld);
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
    contig_body<LOGT, NG, SEP>(p, tile, smem_raw, v);
  else
    strided_body<LOGT, KIN>(p, o, cb, smem_raw, ld);
}

template <int LOGT, bool CONTIG, bool KIN, int NG = 0, bool SEP = false>
__global__ void __launch_bounds__(Geo<LOGT>::THREADS, min_blocks<LOGT>())
    k_pass2s_batch(const PassParams<float>* __restrict__ params, const int64_t* __restrict__ tile_start,
                   const int* __restrict__ block_inst, int64_t block_off, uint32_t flags, int khalf) {
  __shared__ __align__(16) unsigned char raw[sizeof(PassParams<float>)];
  batch_body<LOGT, CONTIG, KIN, NG, SEP>(params, tile_start, block_inst, block_off + blockIdx.x, flags, khalf, raw);
}

static_assert(Geo<3>::SMEM <= kPass2sSmem && Geo<4>::SMEM == kPass2sSmem, "host copy of the size");

}  // namespace p2s
}  // namespace wp
