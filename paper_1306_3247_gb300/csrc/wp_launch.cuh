// Host launchers of the device kernels for one precision (included by the
// per-precision translation units).
#pragma once

#include <mutex>

#include "wp_kernels.cuh"

namespace wp {

static inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

template <class T>
int pass_smem_limit_set(size_t smem) {
  cudaError_t e = (cudaError_t)fixed_smem_limit_set<T>(smem);
  if (e == cudaSuccess) e = (cudaError_t)fixed_obs_smem_limit_set<T>(smem);
  if (e == cudaSuccess) e = (cudaError_t)fixed_grid_smem_limit_set<T>(smem);
  if (e == cudaSuccess) e = (cudaError_t)fixed_grid_obs_smem_limit_set<T>(smem);
  const int a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pass<T, 8, false>, (cudaFuncAttribute)a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pass<T, 8, true>, (cudaFuncAttribute)a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pass<T, 16, false>, (cudaFuncAttribute)a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pass<T, 16, true>, (cudaFuncAttribute)a, (int)smem);
  return cuda_status(e);
}

template <class T>
int res1d_smem_limit_set(size_t smem) {
  cudaError_t e = cudaSuccess;
  const int a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_res1d<T, 8, 256>, (cudaFuncAttribute)a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_res1d<T, 16, 512>, (cudaFuncAttribute)a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_res1d<T, 16, 1024>, (cudaFuncAttribute)a, (int)smem);
  if (e == cudaSuccess) e = (cudaError_t)res1d_fixed_smem_limit_set<T>(smem);
  return cuda_status(e);
}

// p.fixed selects the fixed-size kernel (n = 64..1024, 2048-element tiles, 256 threads),
// with partial sums when they are positions on the contiguous axis or momenta on a
// strided one; otherwise p.ept selects the run-time variant (8 elements per thread: <= 256 threads;
// 16: <= 512).
template <class T>
int launch_pass(const PassParams<T>& p, int64_t ntiles, size_t smem, void* stream) {
  const bool obs = (p.flags & (F_OBS_POS | F_OBS_MOM)) != 0;
  const dim3 grid((unsigned)ntiles), block(p.nthreads);
  cudaStream_t st = (cudaStream_t)stream;
  if constexpr (!std::is_same<T, double>::value) {
    if (pass256_applies<T>(p)) return launch_pass256<T>(p, stream);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (pass2s_applies(p)) return launch_pass2s(p, stream);
  }
  if (p.fixed) {
    if (p.nthreads != 256 || p.logC != 11 - p.logn) return (int)cudaErrorInvalidConfiguration;
    const bool contig = p.log_inner == 0;
    // a static grid potential enters the potential phase and the position sums
    const bool use_grid = (p.grid_rec && (p.flags & F_PHASE)) || (p.grid_v && (p.flags & F_OBS_POS));
    if (use_grid) {
      if (contig && !(p.flags & F_OBS_MOM))
        return obs ? launch_fixed_grid_obs<T>(p, grid.x, smem, stream) : launch_fixed_grid<T>(p, grid.x, smem, stream);
    } else {
      if (!obs) return launch_fixed<T>(p, grid.x, smem, stream);
      // the fixed variant sums positions on the contiguous axis, momenta on a strided one
      if ((contig && !(p.flags & F_OBS_MOM)) || (!contig && !(p.flags & F_OBS_POS)))
        return launch_fixed_obs<T>(p, grid.x, smem, stream);
    }
  }
  if (p.ept == 8 && p.nthreads <= 256) {
    if (obs)
      k_pass<T, 8, true><<<grid, block, smem, st>>>(p);
    else
      k_pass<T, 8, false><<<grid, block, smem, st>>>(p);
  } else if (p.ept == 16 && p.nthreads <= 512) {
    if (obs)
      k_pass<T, 16, true><<<grid, block, smem, st>>>(p);
    else
      k_pass<T, 16, false><<<grid, block, smem, st>>>(p);
  } else {
    return (int)cudaErrorInvalidConfiguration;
  }
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_prep(const PrepParams<T>& p, void* stream) {
  // 64-thread blocks over the entries of all axes: the FP64 work spreads over SMs
  int64_t nall = 0;
  for (int d = 0; d < p.g.ndim; d++) nall += p.n[d];
  int64_t blocks = (nall + 63) / 64;
  if (blocks < 1) blocks = 1;
  if (blocks > 512) blocks = 512;
  k_prep<T><<<(unsigned)blocks, 64, 0, (cudaStream_t)stream>>>(p);
  return cuda_status(cudaGetLastError());
}

// p.ept: 8 elements per thread (<= 256 threads) or 16 (<= 1024 threads).
template <class T>
int launch_res1d(const Res1dParams<T>& p, size_t smem, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (p.fixed) return launch_res1d_fixed<T>(p, smem, stream);
  if (p.ept == 8 && p.nthreads <= 256)
    k_res1d<T, 8, 256><<<1, p.nthreads, smem, st>>>(p);
  else if (p.ept == 16 && p.nthreads <= 512)
    k_res1d<T, 16, 512><<<1, p.nthreads, smem, st>>>(p);
  else if (p.ept == 16 && p.nthreads <= 1024)
    k_res1d<T, 16, 1024><<<1, p.nthreads, smem, st>>>(p);
  else
    return (int)cudaErrorInvalidConfiguration;
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_static_phase(const StaticPhaseParams<T>& p, void* stream) {
  int64_t blocks = (p.n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks > 0) k_static_phase<T><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p);
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_grid_phase(const GridPhaseParams<T>& p, void* stream) {
  int64_t blocks = (p.n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks > 0) k_grid_phase<T><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p);
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_expect(const ExpectParams<T>& p, int nblocks, double dv, double* out, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  k_expect_partial<T><<<(unsigned)nblocks, 256, 0, st>>>(p);
  k_expect_final<T><<<1, 256, 0, st>>>(p.partial, nblocks, dv, out);
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_convert(const ConvParams<T>& p, void* stream) {
  const int64_t blocks = (p.n + 255) / 256;
  if (blocks > 0) k_convert<T><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p);
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_gaussian(const GaussParams<T>& p, int64_t n, void* stream) {
  int64_t ab = (p.nsum + 255) / 256;
  if (ab > 96) ab = 96;
  if (ab > 0) k_gaussian_axes<T><<<(unsigned)ab, 256, 0, (cudaStream_t)stream>>>(p);
  const int64_t blocks = (n + 255) / 256;
  if (blocks > 0) k_gaussian<T><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p, n);
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_lines(const LinesParams<T>& p, void* stream) {
  int64_t blocks = (p.nlines + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks > 0) k_lines<T><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p);
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_pass_batch(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst, int logn,
                      int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, size_t smem, void* stream) {
  // the two-stage complex64 kernels of 256-point lines have a class of their own
  if constexpr (std::is_same<T, float>::value) {
    if (logn >= kBatchClassP2S && logn < kBatchClassP2S + 200)
      return launch_pass2s_batch(params, tile_start, block_inst, 6 + (logn - kBatchClassP2S) / 100,
                                 (logn - kBatchClassP2S) % 100, block_off, nblocks, flags, khalf, stream);
  }
  if constexpr (!std::is_same<T, double>::value) {
    if (logn >= kBatchClassP256 && logn < kBatchClassP256 + 6)
      return launch_pass256_batch<T>(params, tile_start, block_inst, logn - kBatchClassP256, block_off, nblocks,
                                     flags, khalf, stream);
  }
  // the contiguous pass carries the potential phase, the strided one the kinetic factor
  if ((flags & F_KIN) == 0)
    return launch_pass_batch_contig<T>(params, tile_start, block_inst, logn, block_off, nblocks, flags, khalf, smem,
                                       stream);
  return launch_pass_batch_strided<T>(params, tile_start, block_inst, logn, block_off, nblocks, flags, khalf, smem,
                                      stream);
}

template <class T>
int launch_lines_batch(const LinesParams<T>* params, int ninst, int64_t max_lines, void* stream) {
  int64_t bx = (max_lines + 255) / 256;
  if (bx > 64) bx = 64;
  if (ninst > 0 && bx > 0) k_lines_batch<T><<<dim3((unsigned)bx, (unsigned)ninst), 256, 0, (cudaStream_t)stream>>>(params);
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_prep_batch(const PrepParams<T>* params, int ninst, int step_add, double shift_dt, double tau_dt,
                      void* stream) {
  if (ninst > 0)
    k_prep_batch<T><<<(unsigned)ninst, 256, 0, (cudaStream_t)stream>>>(params, step_add, shift_dt, tau_dt);
  return cuda_status(cudaGetLastError());
}

template <class T>
int launch_res1d_batch(const Res1dParams<T>* params, int ninst, int nthreads, int ept, int64_t nsteps, size_t smem,
                       void* stream) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    attr = cudaFuncSetAttribute(k_res1d_batch<T, 8, 256>, a, 200 * 1024);
    if (attr == cudaSuccess) attr = cudaFuncSetAttribute(k_res1d_batch<T, 16, 512>, a, 200 * 1024);
    if (attr == cudaSuccess) attr = cudaFuncSetAttribute(k_res1d_batch<T, 16, 1024>, a, 200 * 1024);
  });
  if (attr != cudaSuccess) return (int)attr;
  if (ninst <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (ept == 8 && nthreads <= 256)
    k_res1d_batch<T, 8, 256><<<(unsigned)ninst, nthreads, smem, st>>>(params, nsteps);
  else if (ept == 16 && nthreads <= 512)
    k_res1d_batch<T, 16, 512><<<(unsigned)ninst, nthreads, smem, st>>>(params, nsteps);
  else if (ept == 16 && nthreads <= 1024)
    k_res1d_batch<T, 16, 1024><<<(unsigned)ninst, nthreads, smem, st>>>(params, nsteps);
  else
    return (int)cudaErrorInvalidConfiguration;
  return cuda_status(cudaGetLastError());
}

#define WP_INSTANTIATE(T)                                                         \
  template int pass_smem_limit_set<T>(size_t);                                    \
  template int res1d_smem_limit_set<T>(size_t);                                   \
  template int launch_pass<T>(const PassParams<T>&, int64_t, size_t, void*);     \
  template int launch_prep<T>(const PrepParams<T>&, void*);                       \
  template int launch_res1d<T>(const Res1dParams<T>&, size_t, void*);            \
  template int launch_convert<T>(const ConvParams<T>&, void*);                    \
  template int launch_static_phase<T>(const StaticPhaseParams<T>&, void*);        \
  template int launch_grid_phase<T>(const GridPhaseParams<T>&, void*);            \
  template int launch_expect<T>(const ExpectParams<T>&, int, double, double*, void*); \
  template int launch_gaussian<T>(const GaussParams<T>&, int64_t, void*);        \
  template int launch_lines<T>(const LinesParams<T>&, void*);                    \
  template int launch_pass_batch<T>(const PassParams<T>*, const int64_t*, const int*, int, int64_t, int64_t, uint32_t, \
                                    int, size_t, void*);                         \
  template int launch_prep_batch<T>(const PrepParams<T>*, int, int, double, double, void*);                    \
  template int launch_lines_batch<T>(const LinesParams<T>*, int, int64_t, void*);                              \
  template int launch_res1d_batch<T>(const Res1dParams<T>*, int, int, int, int64_t, size_t, void*);

}  // namespace wp
