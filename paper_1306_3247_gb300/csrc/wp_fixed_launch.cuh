// Host launchers of the fixed-size pass kernels (n = 64..1024 points per line,
// 2048-element tiles, 256 threads), shared by the per-precision translation units
// wp_fixed_*.cu. OBS selects the variant that also forms the observable partial sums.
#pragma once

#include "wp_kernels.cuh"

namespace wp {
namespace fixed_detail {

template <class T, bool OBS, int LOGN>
void launch_n(const PassParams<T>& p, unsigned ntiles, size_t smem, cudaStream_t st) {
  if (p.log_inner == 0)
    k_pass_fixed<T, LOGN, true, OBS><<<ntiles, 256, smem, st>>>(p);
  else
    k_pass_fixed<T, LOGN, false, OBS><<<ntiles, 256, smem, st>>>(p);
}

template <class T, bool OBS, int LOGN>
cudaError_t set_limit(int smem) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_pass_fixed<T, LOGN, true, OBS>, a, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pass_fixed<T, LOGN, false, OBS>, a, smem);
  return e;
}

template <class T, bool OBS>
int launch(const PassParams<T>& p, unsigned ntiles, size_t smem, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  switch (p.logn) {
    case 6:
      launch_n<T, OBS, 6>(p, ntiles, smem, st);
      break;
    case 7:
      launch_n<T, OBS, 7>(p, ntiles, smem, st);
      break;
    case 8:
      launch_n<T, OBS, 8>(p, ntiles, smem, st);
      break;
    case 9:
      launch_n<T, OBS, 9>(p, ntiles, smem, st);
      break;
    case 10:
      launch_n<T, OBS, 10>(p, ntiles, smem, st);
      break;
    default:
      return (int)cudaErrorInvalidConfiguration;
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

template <class T, bool OBS>
int limit(size_t smem) {
  cudaError_t e = set_limit<T, OBS, 6>((int)smem);
  if (e == cudaSuccess) e = set_limit<T, OBS, 7>((int)smem);
  if (e == cudaSuccess) e = set_limit<T, OBS, 8>((int)smem);
  if (e == cudaSuccess) e = set_limit<T, OBS, 9>((int)smem);
  if (e == cudaSuccess) e = set_limit<T, OBS, 10>((int)smem);
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace fixed_detail
}  // namespace wp

// One translation unit per (precision, variant) so that they compile in parallel.
#define WP_FIXED_TU(T, OBS, LAUNCH, LIMIT)                                                  \
  namespace wp {                                                                            \
  template <>                                                                               \
  int LAUNCH<T>(const PassParams<T>& p, unsigned ntiles, size_t smem, void* stream) {       \
    return fixed_detail::launch<T, OBS>(p, ntiles, smem, stream);                           \
  }                                                                                         \
  template <>                                                                               \
  int LIMIT<T>(size_t smem) {                                                               \
    return fixed_detail::limit<T, OBS>(smem);                                               \
  }                                                                                         \
  }
