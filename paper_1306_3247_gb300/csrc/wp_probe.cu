// Arithmetic-rate probe: the FP64 and FP32 fused multiply-add throughput of the device.
//
// The paper has no counterpart of this entry point. It measures the rate that bounds the
// native FP64 form of the split step on GB300 (whose FP64 pipe, not HBM, sets the pace of
// a complex128 pass), so that a roofline fraction of that form can be stated against a
// rate measured on the same device in the same run.
//
// Method: every thread runs 8 independent FMA chains x <- x b + a (b just below 1, so the
// values stay bounded), enough warps per SM to cover the pipe latency (8 blocks of 256
// threads per SM), timed with CUDA events around a second launch (the first warms up).
// One chain step is one FMA = 2 floating-point operations.
//
// The phase-factor accuracy probe evaluates the complex64 tables' float-float cosine and
// sine (wp_phase_ff.cuh) against the FP64 sincos on a grid of arguments.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "wavepacket_gpu.h"
#include "wp_phase_ff.cuh"

namespace {

__device__ double g_probe_sink[2];

template <class T>
__global__ void __launch_bounds__(256) k_probe_fma(T a, T b, int iters, T* sink) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = a * (T)(threadIdx.x + 1 + k);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = fma(x[k], b, a);
  }
  T s = x[0];
#pragma unroll
  for (int k = 1; k < 8; k++) s += x[k];
  // never true for these inputs: it keeps the chains from being removed
  if (s == (T)-1) sink[0] = s;
}

// Largest |cos - cos_ref| or |sin - sin_ref| over arguments amax (2 (i + 1/2)/n - 1),
// i < n, as the bit pattern of a non-negative double (such patterns order like the values).
__global__ void __launch_bounds__(256) k_probe_phase_ff(int64_t n, double amax, unsigned long long* worst_bits) {
  double worst = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double th = amax * (2.0 * ((double)i + 0.5) / (double)n - 1.0);
    wp::ff c, s;
    wp::cis_ff(th, c, s);
    double sd, cd;
    sincos(th, &sd, &cd);
    const double e = fmax(fabs(((double)c.hi + (double)c.lo) - cd), fabs(((double)s.hi + (double)s.lo) - sd));
    worst = fmax(worst, e);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) atomicMax(worst_bits, (unsigned long long)__double_as_longlong(worst));
}

}  // namespace

extern "C" {

// See include/wavepacket_gpu.h for the contract.
wp_status wp_probe_phase_ff(int64_t n, double amax, void* stream, double* max_err) {
  if (!max_err || n < 1 || !(amax > 0.0) || !std::isfinite(amax)) return WP_EINVAL;
  *max_err = 0.0;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* d = nullptr;
  (void)cudaGetLastError();
  if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return WP_ECUDA;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    const int64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < 4096 ? want : 4096);
    k_probe_phase_ff<<<blocks, 256, 0, st>>>(n, amax, d);
    e = cudaGetLastError();
  }
  unsigned long long bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return WP_ECUDA;
  double v;
  static_assert(sizeof(v) == sizeof(bits), "double and its bit pattern");
  memcpy(&v, &bits, sizeof(v));
  *max_err = v;
  return WP_OK;
}

// See include/wavepacket_gpu.h for the contract.
wp_status wp_probe_fma_rate(int32_t fp64, void* stream, double* tflops) {
  if (!tflops) return WP_EINVAL;
  *tflops = 0.0;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WP_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WP_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  void* sink = nullptr;
  if (cudaGetSymbolAddress(&sink, g_probe_sink) != cudaSuccess) return WP_ECUDA;
  const unsigned blocks = (unsigned)nsm * 8u;
  // about 0.1 s per launch on GB300: FP64 ~0.6e12 FMA/s, FP32 ~35e12 FMA/s
  const int iters = fp64 ? 20000 : 1000000;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return WP_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return WP_ECUDA;
  }
  (void)cudaGetLastError();
  for (int rep = 0; rep < 2; rep++) {
    if (rep == 1) cudaEventRecord(e0, st);
    if (fp64)
      k_probe_fma<double><<<blocks, 256, 0, st>>>(1e-3, 0.999999, iters, (double*)sink);
    else
      k_probe_fma<float><<<blocks, 256, 0, st>>>(1e-3f, 0.9999f, iters, (float*)sink);
  }
  cudaEventRecord(e1, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return WP_ECUDA;
  const double fmas = (double)blocks * 256.0 * 8.0 * (double)iters;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return WP_OK;
}

}  // extern "C"
