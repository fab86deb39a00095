// Allocation-free position moments of a caller-owned complex128 state.
//
// Some callers cannot call cudaMalloc: a host application whose device memory is held
// entirely by its own pool (a framework caching allocator, or a serving process that
// reserved its HBM budget up front), code running in a callback where the host forbids
// allocation, or a loop that cannot afford the implicit device synchronisation an
// allocation may cause. wp_moments_noalloc serves them: it reduces the state into a
// file-scope device array instead of a scratch buffer of the handle, and allocates
// nothing. The paper has no counterpart of this entry point.
//
// The array (g_moment_scratch, 256 KiB + one record) lives in every device that loads the
// library until the process exits. Its size bounds the problem: at most
// kMaxBlocks x kPointsPerBlock = 16,777,216 grid points (e.g. 256^3).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "wavepacket_gpu.h"

namespace {

constexpr int kMaxBlocks = 4096;
constexpr int64_t kPointsPerBlock = 4096;
constexpr int kSlots = 8;  // sum |psi|^2, sum x_d |psi|^2 (3), sum x_d^2 |psi|^2 (3), unused
constexpr int kThreads = 256;

// Partial sums of every block, then the final record (8 doubles). Every slot a call reads
// is written earlier in the same call, so nothing has to start at zero; the contents of the
// previous call are simply overwritten.
static __device__ __align__(256) double g_moment_scratch[kMaxBlocks * kSlots + kSlots];

struct MomentGeom {
  int32_t ndim;
  int64_t n[3];
  double xmin[3], dx[3];
  double dv;
  int64_t npoints;
};

__device__ __forceinline__ void block_sum8(double (&acc)[kSlots], double* out, double (*red)[kSlots]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kSlots; q++) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < kSlots) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; w++) v += red[w][threadIdx.x];
    out[threadIdx.x] = v;
  }
}

// Block b sums the points [b P, (b+1) P) in a fixed order and writes its slots.
__global__ void __launch_bounds__(kThreads) k_moments_partial(const double2* __restrict__ psi, MomentGeom g,
                                                             double* scratch) {
  __shared__ double red[kThreads / 32][kSlots];
  double acc[kSlots];
#pragma unroll
  for (int q = 0; q < kSlots; q++) acc[q] = 0.0;
  const int64_t begin = (int64_t)blockIdx.x * kPointsPerBlock;
  int64_t end = begin + kPointsPerBlock;
  if (end > g.npoints) end = g.npoints;
  for (int64_t idx = begin + threadIdx.x; idx < end; idx += kThreads) {
    const double2 v = psi[idx];
    const double rho = v.x * v.x + v.y * v.y;
    acc[0] += rho;
    int64_t r = idx;
    for (int d = g.ndim - 1; d >= 0; d--) {
      const int64_t i = r % g.n[d];
      r /= g.n[d];
      const double x = g.xmin[d] + (double)i * g.dx[d];
      acc[1 + d] += x * rho;
      acc[4 + d] += x * x * rho;
    }
  }
  block_sum8(acc, scratch + (int64_t)blockIdx.x * kSlots, red);
}

// One block: fixed-order sum of the block partials into the record at the array's tail:
// norm, <x_d> (3), <x_d^2> (3).
__global__ void __launch_bounds__(kThreads) k_moments_final(MomentGeom g, int nblocks, double* scratch) {
  __shared__ double red[kThreads / 32][kSlots];
  __shared__ double tot[kSlots];
  double acc[kSlots];
#pragma unroll
  for (int q = 0; q < kSlots; q++) acc[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
    for (int q = 0; q < kSlots; q++) acc[q] += scratch[(int64_t)b * kSlots + q];
  block_sum8(acc, tot, red);
  __syncthreads();
  if (threadIdx.x == 0) {
    double* rec = scratch + (int64_t)kMaxBlocks * kSlots;
    rec[0] = sqrt(tot[0] * g.dv);
    for (int d = 0; d < 3; d++) {
      rec[1 + d] = tot[1 + d] * g.dv;
      rec[4 + d] = tot[4 + d] * g.dv;
    }
    rec[7] = 0.0;
  }
}

std::mutex g_setup_mutex;
void* g_scratch_addr[64] = {};  // device address of g_moment_scratch, per device ordinal
// The last error message of the calling thread: a call on another thread never replaces
// (and so never frees) the string a caller is reading.
thread_local std::string g_noalloc_err;

wp_status noalloc_fail(wp_status st, const std::string& msg) {
  g_noalloc_err = msg;
  return st;
}

}  // namespace

extern "C" {

// See include/wavepacket_gpu.h for the contract.
wp_status wp_moments_noalloc(const wp_problem* problem, const void* psi_dev, void* stream, wp_obs* out) {
  if (!problem || !psi_dev || !out) return noalloc_fail(WP_EINVAL, "NULL argument");
  if (problem->ndim < 1 || problem->ndim > 3) return noalloc_fail(WP_EUNSUPPORTED, "ndim must be 1, 2 or 3");
  MomentGeom g{};
  g.ndim = problem->ndim;
  g.dv = 1.0;
  g.npoints = 1;
  for (int d = 0; d < 3; d++) {
    g.n[d] = d < problem->ndim ? problem->n[d] : 1;
    if (g.n[d] < 1) return noalloc_fail(WP_EINVAL, "grid extents must be >= 1");
    g.xmin[d] = d < problem->ndim ? problem->xmin[d] : 0.0;
    g.dx[d] = d < problem->ndim ? problem->L[d] / (double)problem->n[d] : 1.0;
    if (d < problem->ndim) g.dv *= g.dx[d];
    if (g.npoints > ((int64_t)1 << 40) / g.n[d]) return noalloc_fail(WP_EUNSUPPORTED, "grid too large");
    g.npoints *= g.n[d];
  }
  const int64_t nblocks = (g.npoints + kPointsPerBlock - 1) / kPointsPerBlock;
  if (nblocks > kMaxBlocks) {
    return noalloc_fail(WP_EUNSUPPORTED,
                        "wp_moments_noalloc: the state has " + std::to_string(g.npoints) +
                            " points; the allocation-free reduction holds at most " +
                            std::to_string((int64_t)kMaxBlocks * kPointsPerBlock) + " (its fixed device array)");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(WP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return noalloc_fail(WP_EUNSUPPORTED, "device ordinal >= 64");
  double* scratch = nullptr;
  {
    // First call on this device (with it current): look up the array's device address.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_moment_scratch);
      if (e != cudaSuccess || !p)
        return noalloc_fail(WP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = (double*)g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  // Clear an earlier, non-sticky launch error so that the checks below see only this
  // call's launches; a launch that fails (no kernel image for the device, a stream of
  // another device) must not let the copy below return the previous call's record.
  (void)cudaGetLastError();
  k_moments_partial<<<(unsigned)nblocks, kThreads, 0, st>>>((const double2*)psi_dev, g, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(WP_ECUDA, std::string("moments launch: ") + cudaGetErrorString(e));
  k_moments_final<<<1, kThreads, 0, st>>>(g, (int)nblocks, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(WP_ECUDA, std::string("moments launch: ") + cudaGetErrorString(e));
  double rec[kSlots];
  e = cudaMemcpyAsync(rec, scratch + (int64_t)kMaxBlocks * kSlots, sizeof(rec), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(WP_ECUDA, std::string("moments: ") + cudaGetErrorString(e));
  wp_obs o{};
  o.t = problem->t0;
  o.norm = rec[0];
  for (int d = 0; d < 3; d++) {
    o.x[d] = rec[1 + d];
    o.x2[d] = rec[4 + d];
  }
  *out = o;
  return WP_OK;
}

const char* wp_moments_noalloc_error(void) { return g_noalloc_err.c_str(); }

}  // extern "C"
