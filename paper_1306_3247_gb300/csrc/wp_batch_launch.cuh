// Host launcher of the batched pass kernel for one precision and one axis kind
// (contiguous: potential phase; strided: kinetic factor), shared by the translation
// units wp_batch_*.cu, which compile in parallel.
#pragma once

#include "wp_kernels.cuh"

namespace wp {
namespace batch_detail {

template <class T, bool CONTIG>
int launch(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst, int64_t ntiles,
           uint32_t flags, int khalf, size_t smem, void* stream) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_pass_batch<T, CONTIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    if (e != cudaSuccess) return (int)e;
    attr = true;
  }
  if (ntiles > 0)
    k_pass_batch<T, CONTIG><<<(unsigned)ntiles, 256, smem, (cudaStream_t)stream>>>(params, tile_start, block_inst,
                                                                                  flags, khalf);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace batch_detail
}  // namespace wp

#define WP_BATCH_TU(T, CONTIG, NAME)                                                                    \
  namespace wp {                                                                                        \
  template <>                                                                                           \
  int NAME<T>(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst,            \
              int64_t ntiles, uint32_t flags, int khalf, size_t smem, void* stream) {                   \
    return batch_detail::launch<T, CONTIG>(params, tile_start, block_inst, ntiles, flags, khalf, smem,  \
                                           stream);                                                     \
  }                                                                                                     \
  }
