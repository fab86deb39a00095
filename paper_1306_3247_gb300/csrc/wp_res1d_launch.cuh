// Host launchers of the fixed-length resident-line kernels (n = 2^8 .. 2^14, n / EPT
// threads), shared by the per-precision translation units wp_res1d_*.cu.
#pragma once

#include "wp_kernels.cuh"

namespace wp {
namespace res1d_detail {

// 16-byte elements: lines of at most 2^13 points (the longest a handle accepts)
template <class T, int LOGN>
constexpr bool supported() {
  return sizeof(cx<T>) == 8 || LOGN <= 13;
}

template <class T, int LOGN>
cudaError_t launch_n(const Res1dParams<T>& p, size_t smem, cudaStream_t st) {
  if constexpr (supported<T, LOGN>()) {
    constexpr int EPT = wp_res1d_fixed_ept(LOGN);
    k_res1d_fixed<T, LOGN, EPT><<<1, (1 << LOGN) / EPT, smem, st>>>(p);
    return cudaGetLastError();
  }
  return cudaErrorInvalidConfiguration;
}

template <class T, int LOGN>
cudaError_t launch_batch_n(const Res1dParams<T>* params, int ninst, int64_t nsteps, size_t smem, cudaStream_t st) {
  if constexpr (supported<T, LOGN>()) {
    constexpr int EPT = wp_res1d_fixed_ept(LOGN);
    k_res1d_fixed_batch<T, LOGN, EPT><<<(unsigned)ninst, (1 << LOGN) / EPT, smem, st>>>(params, nsteps);
    return cudaGetLastError();
  }
  return cudaErrorInvalidConfiguration;
}

template <class T, int LOGN>
cudaError_t set_limit(int smem) {
  if constexpr (supported<T, LOGN>()) {
    constexpr int EPT = wp_res1d_fixed_ept(LOGN);
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_res1d_fixed<T, LOGN, EPT>, a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_res1d_fixed_batch<T, LOGN, EPT>, a, smem);
    return e;
  }
  return cudaSuccess;
}

// Calls F<LOGN>() for LOGN = logn in kRes1dLogMin .. kRes1dLogMax.
template <class F>
bool dispatch(int logn, F&& f) {
  switch (logn) {
    case 8:
      f(std::integral_constant<int, 8>());
      return true;
    case 9:
      f(std::integral_constant<int, 9>());
      return true;
    case 10:
      f(std::integral_constant<int, 10>());
      return true;
    case 11:
      f(std::integral_constant<int, 11>());
      return true;
    case 12:
      f(std::integral_constant<int, 12>());
      return true;
    case 13:
      f(std::integral_constant<int, 13>());
      return true;
    case 14:
      f(std::integral_constant<int, 14>());
      return true;
    default:
      return false;
  }
}

}  // namespace res1d_detail
}  // namespace wp

#define WP_RES1D_TU(T)                                                                                 \
  namespace wp {                                                                                       \
  template <>                                                                                          \
  int launch_res1d_fixed<T>(const Res1dParams<T>& p, size_t smem, void* stream) {                      \
    cudaError_t e = cudaErrorInvalidConfiguration;                                                     \
    res1d_detail::dispatch(p.logn, [&](auto L) {                                                       \
      e = res1d_detail::launch_n<T, decltype(L)::value>(p, smem, (cudaStream_t)stream);                \
    });                                                                                                \
    return e == cudaSuccess ? 0 : (int)e;                                                              \
  }                                                                                                    \
  template <>                                                                                          \
  int launch_res1d_fixed_batch<T>(const Res1dParams<T>* params, int ninst, int logn, int64_t nsteps,  \
                                  size_t smem, void* stream) {                                         \
    if (ninst <= 0) return 0;                                                                          \
    cudaError_t e = cudaErrorInvalidConfiguration;                                                     \
    res1d_detail::dispatch(logn, [&](auto L) {                                                         \
      e = res1d_detail::launch_batch_n<T, decltype(L)::value>(params, ninst, nsteps, smem,             \
                                                              (cudaStream_t)stream);                   \
    });                                                                                                \
    return e == cudaSuccess ? 0 : (int)e;                                                              \
  }                                                                                                    \
  template <>                                                                                          \
  int res1d_fixed_smem_limit_set<T>(size_t smem) {                                                     \
    cudaError_t e = cudaSuccess;                                                                       \
    for (int l = kRes1dLogMin; l <= kRes1dLogMax && e == cudaSuccess; l++)                             \
      res1d_detail::dispatch(l, [&](auto L) { e = res1d_detail::set_limit<T, decltype(L)::value>((int)smem); }); \
    return e == cudaSuccess ? 0 : (int)e;                                                              \
  }                                                                                                    \
  }
