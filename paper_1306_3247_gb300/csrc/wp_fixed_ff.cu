// Fixed-size pass kernels (n = 64..1024 points per line, 2048-element tiles) for the
// float-float complex128-accuracy form, in a translation unit of their own so that they compile in parallel.
#include "wp_kernels.cuh"

namespace wp {

namespace {

template <int LOGN>
void launch_n(const PassParams<ff>& p, unsigned ntiles, size_t smem, cudaStream_t st) {
  if (p.log_inner == 0)
    k_pass_fixed<ff, LOGN, true, false><<<ntiles, 256, smem, st>>>(p);
  else
    k_pass_fixed<ff, LOGN, false, false><<<ntiles, 256, smem, st>>>(p);
}

template <int LOGN>
cudaError_t set_limit(int smem) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_pass_fixed<ff, LOGN, true, false>, a, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pass_fixed<ff, LOGN, false, false>, a, smem);
  return e;
}

}  // namespace

template <>
int launch_fixed<ff>(const PassParams<ff>& p, unsigned ntiles, size_t smem, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  switch (p.logn) {
    case 6:
      launch_n<6>(p, ntiles, smem, st);
      break;
    case 7:
      launch_n<7>(p, ntiles, smem, st);
      break;
    case 8:
      launch_n<8>(p, ntiles, smem, st);
      break;
    case 9:
      launch_n<9>(p, ntiles, smem, st);
      break;
    case 10:
      launch_n<10>(p, ntiles, smem, st);
      break;
    default:
      return (int)cudaErrorInvalidConfiguration;
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

template <>
int fixed_smem_limit_set<ff>(size_t smem) {
  cudaError_t e = set_limit<6>((int)smem);
  if (e == cudaSuccess) e = set_limit<7>((int)smem);
  if (e == cudaSuccess) e = set_limit<8>((int)smem);
  if (e == cudaSuccess) e = set_limit<9>((int)smem);
  if (e == cudaSuccess) e = set_limit<10>((int)smem);
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace wp
