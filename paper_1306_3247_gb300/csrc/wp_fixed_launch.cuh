// Host launchers of the fixed-size pass kernels (n = 64..1024 points per line,
// 2048-element tiles, 256 threads), shared by the per-precision translation units
// wp_fixed_*.cu. OBS selects the variant that also forms the observable partial sums,
// GRID the one that applies a static grid potential (contiguous passes only).
#pragma once

#include <type_traits>

#include "wp_kernels.cuh"

namespace wp {
namespace fixed_detail {

// The kernel of a shape: the FP64 one has its own register bound.
template <class T, int LOGN, bool CONTIG, bool OBS, bool GRID>
constexpr auto kernel_of() {
  if constexpr (std::is_same<T, double>::value)
    return &k_pass_fixed_f64<LOGN, CONTIG, OBS, GRID>;
  else
    return &k_pass_fixed<T, LOGN, CONTIG, OBS, GRID>;
}

template <class T, bool OBS, bool GRID, int LOGN>
cudaError_t launch_n(const PassParams<T>& p, unsigned ntiles, size_t smem, cudaStream_t st) {
  if (p.log_inner == 0) {
    kernel_of<T, LOGN, true, OBS, GRID>()<<<ntiles, 256, smem, st>>>(p);
  } else {
    if constexpr (GRID) return cudaErrorInvalidConfiguration;
    else kernel_of<T, LOGN, false, OBS, false>()<<<ntiles, 256, smem, st>>>(p);
  }
  return cudaGetLastError();
}

template <class T, bool OBS, bool GRID, int LOGN>
cudaError_t set_limit(int smem) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(kernel_of<T, LOGN, true, OBS, GRID>(), a, smem);
  if constexpr (!GRID)
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel_of<T, LOGN, false, OBS, false>(), a, smem);
  return e;
}

template <class T, bool OBS, bool GRID>
int launch(const PassParams<T>& p, unsigned ntiles, size_t smem, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (p.logn) {
    case 6:
      e = launch_n<T, OBS, GRID, 6>(p, ntiles, smem, st);
      break;
    case 7:
      e = launch_n<T, OBS, GRID, 7>(p, ntiles, smem, st);
      break;
    case 8:
      e = launch_n<T, OBS, GRID, 8>(p, ntiles, smem, st);
      break;
    case 9:
      e = launch_n<T, OBS, GRID, 9>(p, ntiles, smem, st);
      break;
    case 10:
      e = launch_n<T, OBS, GRID, 10>(p, ntiles, smem, st);
      break;
    default:
      return (int)cudaErrorInvalidConfiguration;
  }
  return e == cudaSuccess ? 0 : (int)e;
}

template <class T, bool OBS, bool GRID>
int limit(size_t smem) {
  cudaError_t e = set_limit<T, OBS, GRID, 6>((int)smem);
  if (e == cudaSuccess) e = set_limit<T, OBS, GRID, 7>((int)smem);
  if (e == cudaSuccess) e = set_limit<T, OBS, GRID, 8>((int)smem);
  if (e == cudaSuccess) e = set_limit<T, OBS, GRID, 9>((int)smem);
  if (e == cudaSuccess) e = set_limit<T, OBS, GRID, 10>((int)smem);
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace fixed_detail
}  // namespace wp

// One translation unit per (precision, variant) so that they compile in parallel.
#define WP_FIXED_TU(T, OBS, GRID, LAUNCH, LIMIT)                                            \
  namespace wp {                                                                            \
  template <>                                                                               \
  int LAUNCH<T>(const PassParams<T>& p, unsigned ntiles, size_t smem, void* stream) {       \
    return fixed_detail::launch<T, OBS, GRID>(p, ntiles, smem, stream);                     \
  }                                                                                         \
  template <>                                                                               \
  int LIMIT<T>(size_t smem) {                                                               \
    return fixed_detail::limit<T, OBS, GRID>(smem);                                         \
  }                                                                                         \
  }
