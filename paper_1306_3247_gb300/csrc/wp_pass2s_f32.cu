// Host launchers of the two-stage complex64 kernels for 64- and 128-point lines
// (wp_pass2s.cuh).
#include "wp_pass2s.cuh"

namespace wp {

namespace {

template <int LOGT, int NG>
void launch_contig_ng(const PassParams<float>& p, unsigned blocks, cudaStream_t st) {
  using G = p2s::Geo<LOGT>;
  if (p.sep)
    p2s::k_pass2s_contig<LOGT, NG, true><<<blocks, G::THREADS, G::SMEM, st>>>(p);
  else
    p2s::k_pass2s_contig<LOGT, NG, false><<<blocks, G::THREADS, G::SMEM, st>>>(p);
}

template <int LOGT>
int launch_t(const PassParams<float>& p, cudaStream_t st) {
  using G = p2s::Geo<LOGT>;
  int lntot = 0;
  for (int d = 0; d < p.g.ndim; d++) lntot += p.g.ln[d];
  const unsigned blocks = (unsigned)(int64_t(1) << (lntot - G::LOGN - G::LOGLINES));
  if (p.log_inner == 0) {
    const int ng = (p.flags & F_PHASE) ? p.ngauss : 0;
    PassParams<float> q = p;
    q.sep = ((p.flags & F_PHASE) && p.sep) ? 1 : 0;
    if (ng >= 2)
      launch_contig_ng<LOGT, 2>(q, blocks, st);
    else if (ng == 1)
      launch_contig_ng<LOGT, 1>(q, blocks, st);
    else
      launch_contig_ng<LOGT, 0>(q, blocks, st);
  } else if (p.flags & F_KIN) {
    p2s::k_pass2s_strided<LOGT, true><<<blocks, G::THREADS, G::SMEM, st>>>(p);
  } else {
    p2s::k_pass2s_strided<LOGT, false><<<blocks, G::THREADS, G::SMEM, st>>>(p);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

template <int LOGT>
int launch_batch_t(const PassParams<float>* params, const int64_t* tile_start, const int* block_inst, int variant,
                   int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, cudaStream_t st) {
  using G = p2s::Geo<LOGT>;
  if (nblocks > 0) {
    auto go = [&](auto kern) {
      kern<<<(unsigned)nblocks, G::THREADS, G::SMEM, st>>>(params, tile_start, block_inst, block_off, flags, khalf);
    };
    if (flags & F_KIN) {
      go(p2s::k_pass2s_batch<LOGT, false, true>);
    } else if (variant < 0) {
      go(p2s::k_pass2s_batch<LOGT, false, false>);
    } else {
      const int ng = (flags & F_PHASE) ? variant >> 1 : 0;
      const bool sep = (flags & F_PHASE) && (variant & 1);
      if (ng == 0)
        sep ? go(p2s::k_pass2s_batch<LOGT, true, false, 0, true>) : go(p2s::k_pass2s_batch<LOGT, true, false, 0, false>);
      else if (ng == 1)
        sep ? go(p2s::k_pass2s_batch<LOGT, true, false, 1, true>) : go(p2s::k_pass2s_batch<LOGT, true, false, 1, false>);
      else
        sep ? go(p2s::k_pass2s_batch<LOGT, true, false, 2, true>) : go(p2s::k_pass2s_batch<LOGT, true, false, 2, false>);
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace

// The two-stage kernels serve a complex64 pass of 64- or 128-point lines when: the
// fixed-shape schedule, no partial sums, no grid potential, and whole tiles (32 lines of
// 64 points or 16 of 128 on a contiguous axis, as many adjacent columns on a strided one).
bool pass2s_applies(const PassParams<float>& p) {
  if (!p.fixed || (p.logn != 6 && p.logn != 7) || !p.W2s) return false;
  if (p.flags & (F_OBS_POS | F_OBS_MOM | F_NO_STORE | F_AUTOCORR)) return false;
  if (p.grid_rec && (p.flags & F_PHASE)) return false;
  int lntot = 0;
  for (int d = 0; d < p.g.ndim; d++) lntot += p.g.ln[d];
  const int loglines = 8 - (p.logn - 3);  // 32 or 16 lines per block
  if (p.log_inner == 0) return lntot - p.logn >= loglines && !(p.flags & F_KIN);
  if (p.flags & F_PHASE) return false;
  return p.log_inner >= loglines;
}

int launch_pass2s(const PassParams<float>& p, void* stream) {
  return p.logn == 6 ? launch_t<3>(p, (cudaStream_t)stream) : launch_t<4>(p, (cudaStream_t)stream);
}

int launch_pass2s_batch(const PassParams<float>* params, const int64_t* tile_start, const int* block_inst, int logn,
                        int variant, int64_t block_off, int64_t nblocks, uint32_t flags, int khalf, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  return logn == 6 ? launch_batch_t<3>(params, tile_start, block_inst, variant, block_off, nblocks, flags, khalf, st)
                   : launch_batch_t<4>(params, tile_start, block_inst, variant, block_off, nblocks, flags, khalf, st);
}

}  // namespace wp
