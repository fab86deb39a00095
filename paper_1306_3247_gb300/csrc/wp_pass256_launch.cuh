// Host launchers of the two-stage 256-point pass kernels (wp_pass256.cuh), shared by the
// translation units of the complex64 and float-float forms.
#pragma once

#include <mutex>
#include <type_traits>

#include "wp_pass256.cuh"
#include "wp_pass256_tma.cuh"

namespace wp {
namespace p256_detail {

template <class T>
constexpr bool two_stage_strided() { return std::is_same<T, float>::value; }

// The two-stage kernels serve a pass when: 256 points along the axis, the fixed-shape
// schedule, no grid potential, whole tiles (L lines of a contiguous axis, L adjacent
// columns of a strided one; L = 16 complex64, 8 float-float), and partial sums only in
// complex64: position sums on the contiguous axis, momentum sums after a forward
// transform on a strided one.
template <class T>
bool applies(const PassParams<T>& p) {
  if (!p.fixed || p.logn != p256::kLogN || !p.W256) return false;
  const uint32_t f = p.flags;
  if (f & (F_OBS_POS | F_OBS_MOM | F_NO_STORE | F_AUTOCORR)) {
    if (!std::is_same<T, float>::value || !p.partials) return false;
    if (p.log_inner == 0) {
      if ((f & F_OBS_MOM) || !(f & F_OBS_POS) || p.grid_v) return false;
    } else if ((f & (F_OBS_POS | F_AUTOCORR | F_KIN | F_IFFT)) || !(f & F_OBS_MOM) || !(f & F_FFT)) {
      return false;
    }
  }
  if (p.grid_rec && (f & F_PHASE)) return false;
  int lntot = 0;
  for (int d = 0; d < p.g.ndim; d++) lntot += p.g.ln[d];
  const int lines_log = lntot - p256::kLogN;
  constexpr int LL = p256::Shape<T>::kLogLines;
  if (p.log_inner == 0) return lines_log >= LL && !(p.flags & F_KIN);
  if (p.flags & F_PHASE) return false;  // the potential phase runs on the contiguous axis
  // float-float: measured on the 256^3 job, its two-stage strided passes were slower than
  // the Stockham ones (180 against 155 us FFT-only, 403 against 324 us kinetic: its
  // arithmetic dominates, so the two-stage form saves only 5 % of the instructions, and at
  // 128 registers it runs 16 warps per SM), while its contiguous pass is faster (336
  // against 391 us): float-float takes the two-stage kernels on the contiguous axis only
  if (!two_stage_strided<T>()) return false;
  return p.log_inner >= LL;
}

// The contiguous kernel of the potential's kind: Gaussian terms (0..2), additive terms;
// the variant with position sums for complex64.
template <class T, int NG>
void launch_contig_ng(const PassParams<T>& p, unsigned blocks, cudaStream_t st) {
  constexpr unsigned nt = p256::threads_of<T>();
  if constexpr (std::is_same<T, float>::value) {
    if (p.flags & F_OBS_POS) {
      if (p.sep)
        p256::k_pass256_contig<T, NG, true, true><<<blocks, nt, p256::kSmem, st>>>(p);
      else
        p256::k_pass256_contig<T, NG, false, true><<<blocks, nt, p256::kSmem, st>>>(p);
      return;
    }
  }
  if (p.sep)
    p256::k_pass256_contig<T, NG, true><<<blocks, nt, p256::kSmem, st>>>(p);
  else
    p256::k_pass256_contig<T, NG, false><<<blocks, nt, p256::kSmem, st>>>(p);
}

// Tensor maps of the TMA-staged strided kernel: the state seen as rows of 2^log_inner
// 8-byte points, box 16 x 256, 128-byte swizzle. cuTensorMapEncodeTiled comes from the
// driver through the runtime's entry-point query (no link against the driver library).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiled encode_fn() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
    (void)cudaGetLastError();
  });
  return fn;
}

inline bool tile_map(EncodeTiled enc, const void* base, int log_inner, int lntot, CUtensorMap* m) {
  const cuuint64_t dims[2] = {cuuint64_t(1) << log_inner, cuuint64_t(1) << (lntot - log_inner)};
  const cuuint64_t strides[1] = {(cuuint64_t(1) << log_inner) * 8};
  const cuuint32_t box[2] = {16, 256};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Blocks of a pass launch (one partial row each when it forms sums).
template <class T>
int64_t blocks_of(const PassParams<T>& p) {
  int lntot = 0;
  for (int d = 0; d < p.g.ndim; d++) lntot += p.g.ln[d];
  return int64_t(1) << (lntot - p256::kLogN - p256::Shape<T>::kLogLines);
}

template <class T>
int launch(const PassParams<T>& p, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int lntot = 0;
  for (int d = 0; d < p.g.ndim; d++) lntot += p.g.ln[d];
  const unsigned blocks = (unsigned)(int64_t(1) << (lntot - p256::kLogN - p256::Shape<T>::kLogLines));
  if (p.log_inner == 0) {
    const int ng = (p.flags & F_PHASE) ? p.ngauss : 0;
    PassParams<T> q = p;
    q.sep = ((p.flags & F_PHASE) && p.sep) ? 1 : 0;
    if (ng >= 2)
      launch_contig_ng<T, 2>(q, blocks, st);
    else if (ng == 1)
      launch_contig_ng<T, 1>(q, blocks, st);
    else
      launch_contig_ng<T, 0>(q, blocks, st);
  } else {
    // complex64: the tile moved by the TMA (same arithmetic); the thread-staged kernel
    // where no tensor map can be made
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      const EncodeTiled enc = encode_fn();
      alignas(64) CUtensorMap tin, tout;
      if (enc && tile_map(enc, p.in, p.log_inner, lntot, &tin) && tile_map(enc, p.out, p.log_inner, lntot, &tout)) {
        if (p.flags & F_KIN)
          p256::k_pass256_strided_tma<true><<<blocks, 256, p256::kTmaSmem, st>>>(p, tin, tout);
        else if (p.flags & F_OBS_MOM)
          p256::k_pass256_strided_tma<false, true><<<blocks, 256, p256::kTmaSmem, st>>>(p, tin, tout);
        else
          p256::k_pass256_strided_tma<false><<<blocks, 256, p256::kTmaSmem, st>>>(p, tin, tout);
        done = true;
      }
    }
    if (!done) {
      constexpr unsigned nt = p256::threads_of<T>();
      if (p.flags & F_KIN)
        p256::k_pass256_strided<T, true><<<blocks, nt, p256::kSmem, st>>>(p);
      else if (std::is_same<T, float>::value && (p.flags & F_OBS_MOM))
        p256::k_pass256_strided<T, false, std::is_same<T, float>::value><<<blocks, nt, p256::kSmem, st>>>(p);
      else
        p256::k_pass256_strided<T, false><<<blocks, nt, p256::kSmem, st>>>(p);
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

template <class T>
int launch_batch(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst, int variant,
                 int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (nblocks > 0) {
    const dim3 grid((unsigned)nblocks), block(p256::threads_of<T>());
    auto go = [&](auto kern) { kern<<<grid, block, p256::kSmem, st>>>(params, tile_start, block_inst, block_off, flags,
                                                                      khalf); };
    if (flags & F_KIN) {
      go(p256::k_pass256_batch<T, false, true>);
    } else if (variant < 0) {
      go(p256::k_pass256_batch<T, false, false>);
    } else {
      // contiguous: the class's largest Gaussian-term count and whether any instance has
      // additive terms (an instance without them multiplies by factors that are exactly 1)
      const int ng = (flags & F_PHASE) ? variant >> 1 : 0;
      const bool sep = (flags & F_PHASE) && (variant & 1);
      if (ng == 0)
        sep ? go(p256::k_pass256_batch<T, true, false, 0, true>) : go(p256::k_pass256_batch<T, true, false, 0, false>);
      else if (ng == 1)
        sep ? go(p256::k_pass256_batch<T, true, false, 1, true>) : go(p256::k_pass256_batch<T, true, false, 1, false>);
      else
        sep ? go(p256::k_pass256_batch<T, true, false, 2, true>) : go(p256::k_pass256_batch<T, true, false, 2, false>);
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace p256_detail
}  // namespace wp

#define WP_PASS256_TU(T)                                                                                       \
  namespace wp {                                                                                               \
  template <>                                                                                                  \
  bool pass256_applies<T>(const PassParams<T>& p) {                                                            \
    return p256_detail::applies<T>(p);                                                                         \
  }                                                                                                            \
  template <>                                                                                                  \
  int64_t pass256_blocks<T>(const PassParams<T>& p) {                                                          \
    return p256_detail::blocks_of<T>(p);                                                                       \
  }                                                                                                            \
  template <>                                                                                                  \
  int launch_pass256<T>(const PassParams<T>& p, void* stream) {                                                \
    return p256_detail::launch<T>(p, stream);                                                                  \
  }                                                                                                            \
  template <>                                                                                                  \
  int launch_pass256_batch<T>(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst,   \
                              int variant, int64_t block_off, int64_t nblocks, uint32_t flags, int khalf,      \
                              void* stream) {                                                                  \
    return p256_detail::launch_batch<T>(params, tile_start, block_inst, variant, block_off, nblocks, flags,    \
                                        khalf, stream);                                                        \
  }                                                                                                            \
  }
