// One launch per pass of an uneven batch (the 2-D instances of wp_batch): the blocks of
// the Stockham line-length classes of the pass run in the same grid, each block picking
// its class from the launch's class table, and the per-instance tables and line records
// of the next step (k_prep_batch and k_lines_batch work) run as leading blocks of the
// kinetic pass.
// The kinetic pass reads neither the potential tables nor the line records of the
// potential pass, and the potential pass that read the current ones has completed before
// it starts, so the next step's tables can be written beside it.
#pragma once

#include <mutex>
#include <type_traits>

#include "wp_kernels.cuh"
#include "wp_pass2s.cuh"

namespace wp {

// The per-instance tables of the step (prep_body with the instance's own parameters,
// one block) followed, when `lines`, by the line records of its potential pass.
template <class T>
__device__ __forceinline__ void prep_lines_block(const PrepParams<T>* __restrict__ pp,
                                                 const LinesParams<T>* __restrict__ lp, int inst,
                                                 const MergedLaunch& ml) {
  __shared__ __align__(16) unsigned char raw[sizeof(PrepParams<T>)];
  PrepParams<T>& p = *reinterpret_cast<PrepParams<T>*>(raw);
  const int* src = reinterpret_cast<const int*>(&pp[inst]);
  for (int k = threadIdx.x; k < (int)(sizeof(PrepParams<T>) / sizeof(int)); k += blockDim.x)
    reinterpret_cast<int*>(raw)[k] = src[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    p.step_add = ml.step_add;
    p.t_shift = ml.shift_dt * p.g.dt;
    p.tau = ml.tau_dt * p.g.dt;
  }
  __syncthreads();
  prep_body<T>(p, 0, 1);
  if (!ml.lines) return;
  // the tables and the control block written above are visible to the whole block
  __syncthreads();
  __shared__ __align__(16) unsigned char rawl[sizeof(LinesParams<T>)];
  const int* srcl = reinterpret_cast<const int*>(&lp[inst]);
  for (int k = threadIdx.x; k < (int)(sizeof(LinesParams<T>) / sizeof(int)); k += blockDim.x)
    reinterpret_cast<int*>(rawl)[k] = srcl[k];
  __syncthreads();
  lines_body<T>(*reinterpret_cast<const LinesParams<T>*>(rawl), threadIdx.x, blockDim.x);
}

// The two-stage complex64 body of a 64- (LOGT 3) or 128-point (LOGT 4) class.
template <int LOGT, bool CONTIG>
__device__ __forceinline__ void merged_p2s(int v, const PassParams<float>* __restrict__ params,
                                           const int64_t* __restrict__ tile_start, const int* __restrict__ block_inst,
                                           int64_t blk, uint32_t flags, int khalf, unsigned char* raw) {
  if constexpr (!CONTIG) {
    p2s::batch_body<LOGT, false, true>(params, tile_start, block_inst, blk, flags, khalf, raw);
  } else if (!(flags & F_PHASE)) {
    p2s::batch_body<LOGT, true, false, 0, false>(params, tile_start, block_inst, blk, flags, khalf, raw);
  } else if (v == 1) {
    p2s::batch_body<LOGT, true, false, 0, true>(params, tile_start, block_inst, blk, flags, khalf, raw);
  } else if (v == 2) {
    p2s::batch_body<LOGT, true, false, 1, false>(params, tile_start, block_inst, blk, flags, khalf, raw);
  } else if (v == 3) {
    p2s::batch_body<LOGT, true, false, 1, true>(params, tile_start, block_inst, blk, flags, khalf, raw);
  } else if (v == 4) {
    p2s::batch_body<LOGT, true, false, 2, false>(params, tile_start, block_inst, blk, flags, khalf, raw);
  } else {
    p2s::batch_body<LOGT, true, false, 2, true>(params, tile_start, block_inst, blk, flags, khalf, raw);
  }
}

// Body of class key `key` for block-list entry blk. The merged launch holds the Stockham
// classes of 64-, 128- and 256-point lines (the line lengths of uneven 2-D batches). Each
// class body adds its static shared memory to the kernel's, and the launch's dynamic
// shared memory is the largest class's, so the other classes (longer lines, and the
// two-stage complex64 class with its 39 KB per block) keep launches of their own: with
// them in one grid every block would be sized for the largest, and fewer would fit an SM
// (measured: the complex64 batch 3 % slower with the two-stage class merged in).
template <class T, bool CONTIG>
__device__ __forceinline__ void merged_class_body(int key, const PassParams<T>* __restrict__ params,
                                                  const int64_t* __restrict__ tile_start,
                                                  const int* __restrict__ block_inst, int64_t blk, uint32_t flags,
                                                  int khalf, unsigned char* raw) {
  switch (key) {
    case 6:
      pass_batch_body<T, CONTIG, 6>(params, tile_start, block_inst, blk, flags, khalf, raw);
      break;
    case 7:
      pass_batch_body<T, CONTIG, 7>(params, tile_start, block_inst, blk, flags, khalf, raw);
      break;
    case 8:
      pass_batch_body<T, CONTIG, 8>(params, tile_start, block_inst, blk, flags, khalf, raw);
      break;
    default:
      if constexpr (std::is_same<T, float>::value) {
        // two-stage 64- and 128-point classes; contiguous variant 2 NG + SEP
        const int r = key - kBatchClassP2S, v = r % 100;
        if (r >= 0 && r < 100)
          merged_p2s<3, CONTIG>(v, params, tile_start, block_inst, blk, flags, khalf, raw);
        else if (r >= 100 && r < 200)
          merged_p2s<4, CONTIG>(v, params, tile_start, block_inst, blk, flags, khalf, raw);
      }
      break;
  }
}

template <class T>
constexpr int merged_min_blocks() {
  // complex64: five blocks per SM (the single-class kernels took 32-48 registers); FP64
  // the four of its fixed-shape batched kernels; float-float three
  return std::is_same<T, float>::value ? 5 : (std::is_same<T, ff>::value ? 3 : 4);
}

// CONTIG: the potential pass (axis 1) or the kinetic pass (axis 0). Launch blocks
// 0 .. ml.nprep - 1 form the tables of instance (block); the blocks after them serve the
// classes: ml.nprep + ml.start[c] .. ml.nprep + ml.start[c + 1] - 1 class c (block-list
// entries from ml.list_off[c]). The table blocks come first so that they are dispatched
// first: their work is FP64 (the phase sincos), the pass blocks' FP32 and memory, and
// the two run side by side on the SMs; as trailing blocks they formed the launch's tail
// (ncu: FP64 pipe 37 % busy over the launch). No pass block reads what they write.
template <class T, bool CONTIG>
__global__ void __launch_bounds__(256, merged_min_blocks<T>())
    k_pass_batch_merged(const PassParams<T>* __restrict__ params, const int64_t* __restrict__ tile_start,
                        const int* __restrict__ block_inst, const MergedLaunch ml, uint32_t flags, int khalf,
                        const PrepParams<T>* __restrict__ pp, const LinesParams<T>* __restrict__ lp) {
  if ((int64_t)blockIdx.x < ml.nprep) {
    prep_lines_block<T>(pp, lp, (int)blockIdx.x, ml);
    return;
  }
  const int64_t b = (int64_t)blockIdx.x - ml.nprep;
  __shared__ __align__(16) unsigned char raw[sizeof(PassParams<T>)];
  int c = 0;
  while (c + 1 < ml.ncls && b >= ml.start[c + 1]) c++;
  merged_class_body<T, CONTIG>(ml.key[c], params, tile_start, block_inst, ml.list_off[c] + (b - ml.start[c]), flags,
                               khalf, raw);
}

// Host launcher (one translation unit per precision and pass kind).
template <class T, bool CONTIG>
int launch_merged(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst,
                  const MergedLaunch& ml, uint32_t flags, int khalf, const PrepParams<T>* pp,
                  const LinesParams<T>* lp, size_t smem, void* stream) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_pass_batch_merged<T, CONTIG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                64 * 1024);
  });
  if (attr != cudaSuccess) return (int)attr;
  const int64_t nblocks = ml.start[ml.ncls] + ml.nprep;
  if (nblocks > 0)
    k_pass_batch_merged<T, CONTIG><<<(unsigned)nblocks, 256, smem, (cudaStream_t)stream>>>(
        params, tile_start, block_inst, ml, flags, khalf, pp, lp);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace wp

#define WP_MERGED_TU(T, CONTIG, NAME)                                                                             \
  namespace wp {                                                                                                  \
  template <>                                                                                                     \
  int NAME<T>(const PassParams<T>* params, const int64_t* tile_start, const int* block_inst,                     \
              const MergedLaunch& ml, uint32_t flags, int khalf, const PrepParams<T>* pp,                        \
              const LinesParams<T>* lp, size_t smem, void* stream) {                                             \
    return launch_merged<T, CONTIG>(params, tile_start, block_inst, ml, flags, khalf, pp, lp, smem, stream);     \
  }                                                                                                               \
  }
