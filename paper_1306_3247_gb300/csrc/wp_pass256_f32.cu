// Host launcher of the two-stage complex64 pass kernels for 256-point lines
// (wp_pass256.cuh).
#include "wp_pass256.cuh"

namespace wp {

// The two-stage kernels serve a pass when: complex64, 256 points along the axis, the
// fixed-shape schedule, no partial sums, no grid potential, and whole tiles (16 lines
// of a contiguous axis, 16 adjacent columns of a strided one).
bool pass256_applies(const PassParams<float>& p) {
  if (!p.fixed || p.logn != p256::kLogN || !p.W256) return false;
  if (p.flags & (F_OBS_POS | F_OBS_MOM | F_NO_STORE | F_AUTOCORR)) return false;
  if (p.grid_rec && (p.flags & F_PHASE)) return false;
  int lntot = 0;
  for (int d = 0; d < p.g.ndim; d++) lntot += p.g.ln[d];
  const int lines_log = lntot - p256::kLogN;
  if (p.log_inner == 0) return lines_log >= 4 && !(p.flags & F_KIN);
  if (p.flags & F_PHASE) return false;  // the potential phase runs on the contiguous axis
  return p.log_inner >= 4;
}

int launch_pass256(const PassParams<float>& p, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int lntot = 0;
  for (int d = 0; d < p.g.ndim; d++) lntot += p.g.ln[d];
  const unsigned blocks = (unsigned)(int64_t(1) << (lntot - p256::kLogN - 4));  // 16 lines or columns per block
  if (p.log_inner == 0)
    p256::k_pass256_contig<<<blocks, p256::kThreads, p256::kSmem, st>>>(p);
  else
    if (p.flags & F_KIN)
      p256::k_pass256_strided<true><<<blocks, p256::kThreads, p256::kSmem, st>>>(p);
    else
      p256::k_pass256_strided<false><<<blocks, p256::kThreads, p256::kSmem, st>>>(p);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

int launch_pass256_batch(const PassParams<float>* params, const int64_t* tile_start, const int* block_inst,
                         bool contig, int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (nblocks > 0) {
    if (contig)
      p256::k_pass256_batch<true, false><<<(unsigned)nblocks, p256::kThreads, p256::kSmem, st>>>(
          params, tile_start, block_inst, block_off, flags, khalf);
    else if (flags & F_KIN)
      p256::k_pass256_batch<false, true><<<(unsigned)nblocks, p256::kThreads, p256::kSmem, st>>>(
          params, tile_start, block_inst, block_off, flags, khalf);
    else
      p256::k_pass256_batch<false, false><<<(unsigned)nblocks, p256::kThreads, p256::kSmem, st>>>(
          params, tile_start, block_inst, block_off, flags, khalf);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace wp
