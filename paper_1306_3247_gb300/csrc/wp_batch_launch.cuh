// Host launcher of the batched pass kernel for one precision and one axis kind
// (contiguous: potential phase; strided: kinetic factor), shared by the translation
// units wp_batch_*.cu, which compile in parallel.
#pragma once

#include <mutex>
#include <type_traits>

#include "wp_kernels.cuh"

namespace wp {
namespace batch_detail {

template <class T, bool CONTIG, int LOGN>
int launch_cls(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst, int64_t block_off,
               int64_t nblocks, uint32_t flags, int khalf, size_t smem, cudaStream_t st) {
  // the FP64 kernels of compile-time shape have their own register bound
  constexpr auto kern = [] {
    if constexpr (std::is_same<T, double>::value && LOGN > 0)
      return &k_pass_batch_f64<CONTIG, LOGN>;
    else
      return &k_pass_batch<T, CONTIG, LOGN>;
  }();
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  });
  if (attr != cudaSuccess) return (int)attr;
  if (nblocks > 0)
    kern<<<(unsigned)nblocks, 256, smem, st>>>(params, tile_start, block_inst, block_off, flags, khalf);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

// One launch for the class of line length 2^logn (6..10: fixed-size kernels; other: run-time shape).
template <class T, bool CONTIG>
int launch(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst, int logn,
           int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, size_t smem, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  switch (logn) {
    case 6:
      return launch_cls<T, CONTIG, 6>(params, tile_start, block_inst, block_off, nblocks, flags, khalf, smem, st);
    case 7:
      return launch_cls<T, CONTIG, 7>(params, tile_start, block_inst, block_off, nblocks, flags, khalf, smem, st);
    case 8:
      return launch_cls<T, CONTIG, 8>(params, tile_start, block_inst, block_off, nblocks, flags, khalf, smem, st);
    case 9:
      return launch_cls<T, CONTIG, 9>(params, tile_start, block_inst, block_off, nblocks, flags, khalf, smem, st);
    case 10:
      return launch_cls<T, CONTIG, 10>(params, tile_start, block_inst, block_off, nblocks, flags, khalf, smem, st);
    default:
      return launch_cls<T, CONTIG, 0>(params, tile_start, block_inst, block_off, nblocks, flags, khalf, smem, st);
  }
}

}  // namespace batch_detail
}  // namespace wp

#define WP_BATCH_TU(T, CONTIG, NAME)                                                                      \
  namespace wp {                                                                                          \
  template <>                                                                                             \
  int NAME<T>(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst, int logn,   \
              int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, size_t smem, void* stream) { \
    return batch_detail::launch<T, CONTIG>(params, tile_start, block_inst, logn, block_off, nblocks, flags, \
                                           khalf, smem, stream);                                          \
  }                                                                                                       \
  }
