// Host launcher of the two-stage complex64 pass kernels for 256-point lines
// (wp_pass256.cuh).
#include "wp_pass256.cuh"

namespace wp {

namespace {

// The contiguous kernel of the potential's kind: Gaussian terms (0..2), additive terms.
template <int NG>
void launch_contig_ng(const PassParams<float>& p, unsigned blocks, cudaStream_t st) {
  if (p.sep)
    p256::k_pass256_contig<NG, true><<<blocks, p256::kThreads, p256::kSmem, st>>>(p);
  else
    p256::k_pass256_contig<NG, false><<<blocks, p256::kThreads, p256::kSmem, st>>>(p);
}

void launch_contig(const PassParams<float>& p, unsigned blocks, cudaStream_t st) {
  const int ng = (p.flags & F_PHASE) ? p.ngauss : 0;
  const bool sep = (p.flags & F_PHASE) && p.sep;
  PassParams<float> q = p;
  q.sep = sep ? 1 : 0;
  if (ng >= 2)
    launch_contig_ng<2>(q, blocks, st);
  else if (ng == 1)
    launch_contig_ng<1>(q, blocks, st);
  else
    launch_contig_ng<0>(q, blocks, st);
}

}  // namespace

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
    launch_contig(p, blocks, st);
  else
    if (p.flags & F_KIN)
      p256::k_pass256_strided<true><<<blocks, p256::kThreads, p256::kSmem, st>>>(p);
    else
      p256::k_pass256_strided<false><<<blocks, p256::kThreads, p256::kSmem, st>>>(p);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

int launch_pass256_batch(const PassParams<float>* params, const int64_t* tile_start, const int* block_inst,
                         int variant, int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (nblocks > 0) {
    if (flags & F_KIN) {
      p256::k_pass256_batch<false, true><<<(unsigned)nblocks, p256::kThreads, p256::kSmem, st>>>(
          params, tile_start, block_inst, block_off, flags, khalf);
    } else if (variant < 0) {
      p256::k_pass256_batch<false, false><<<(unsigned)nblocks, p256::kThreads, p256::kSmem, st>>>(
          params, tile_start, block_inst, block_off, flags, khalf);
    } else {
      // contiguous: the class's largest Gaussian-term count and whether any instance has
      // additive terms (an instance without them multiplies by factors that are exactly 1)
      const int ng = (flags & F_PHASE) ? variant >> 1 : 0;
      const bool sep = (flags & F_PHASE) && (variant & 1);
      auto go = [&](auto kern) { kern<<<(unsigned)nblocks, p256::kThreads, p256::kSmem, st>>>(
                                     params, tile_start, block_inst, block_off, flags, khalf); };
      if (ng == 0)
        sep ? go(p256::k_pass256_batch<true, false, 0, true>) : go(p256::k_pass256_batch<true, false, 0, false>);
      else if (ng == 1)
        sep ? go(p256::k_pass256_batch<true, false, 1, true>) : go(p256::k_pass256_batch<true, false, 1, false>);
      else
        sep ? go(p256::k_pass256_batch<true, false, 2, true>) : go(p256::k_pass256_batch<true, false, 2, false>);
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace wp
