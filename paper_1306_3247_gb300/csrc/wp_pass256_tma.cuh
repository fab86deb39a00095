// Strided-axis 256-point complex64 pass with its tile moved by the Tensor Memory
// Accelerator: one bulk tensor copy brings the 16 adjacent columns x 256 rows of the tile
// (32 KB) into shared memory and one writes it back, in place of 8 16-byte loads, 16
// shared-memory stores, 16 shared-memory loads and 8 16-byte stores per thread.
//
// The box lands in shared memory row by row (128 bytes per row) with the 128-byte swizzle:
// the 16-byte chunk j of row r sits at chunk j ^ (r mod 8), so that the 16 threads of a
// line, which read one column at 16 rows, hit distinct bank pairs. After the threads have
// read their lines the same region holds the warps' transposes (line-major regions, as in
// k_pass256_strided); the results are written back in the swizzled layout and stored by
// the TMA. The transform, the factors and their order are those of k_pass256_strided, so
// the result is the same bit for bit.
//
// The copy completes on an mbarrier that one thread waits for with a bounded number of
// polls; should it not complete, the kernel records WP_ETIMEOUT in the control block (read
// by wp_run), waits once more (bounded) for the copy and leaves without touching the state.
#pragma once

#include <cuda.h>

#include "wp_pass256.cuh"

namespace wp {
namespace p256 {

constexpr int kTmaBox = 16 * 256 * 8;  // bytes of one tile
constexpr size_t kTmaSmem = kN * sizeof(TwE<float>) + 1024 + (size_t)16 * kLS * sizeof(cx<float>) + 16;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Byte offset of point (row, column c) in the swizzled 128-byte-row layout.
__device__ __forceinline__ uint32_t swz(int row, int c) {
  return (uint32_t)(row * 128 + ((((c >> 1) ^ (row & 7))) << 4) + ((c & 1) << 3));
}

// tm_in / tm_out: 2-D maps of the state seen as rows of 2^log_inner points (8-byte
// elements), box 16 x 256, 128-byte swizzle. Flags and tiles as k_pass256_strided.
// OBS: the momentum sums after the forward transform (and F_NO_STORE), as
// k_pass256_strided<float, false, true>.
template <bool KIN, bool OBS = false>
__global__ void __launch_bounds__(256, Shape<float>::kMinBlocks)
    k_pass256_strided_tma(const PassParams<float> p, const __grid_constant__ CUtensorMap tm_in,
                          const __grid_constant__ CUtensorMap tm_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TwE<float>* s_tw = reinterpret_cast<TwE<float>*>(smem_raw);
  // the tile starts at the first 1024-byte boundary after the twiddles (the swizzle
  // pattern follows the shared-memory address)
  const uint32_t base = smem_u32(smem_raw);
  const uint32_t pad = (1024u - ((base + kN * sizeof(TwE<float>)) & 1023u)) & 1023u;
  unsigned char* tile = smem_raw + kN * sizeof(TwE<float>) + pad;
  const uint32_t tile_s = smem_u32(tile);
  uint64_t* bar = reinterpret_cast<uint64_t*>(tile + (size_t)16 * kLS * sizeof(cx<float>));
  const uint32_t bar_s = smem_u32(bar);
  __shared__ int s_ok;

  int64_t o, cb;
  strided_origin<float>(p.log_inner, blockIdx.x, o, cb);
  const int x = (int)cb, y = (int)(o << kLogN);
  if (threadIdx.x == 0) {
    mbar_init(bar_s, 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar_s, kTmaBox);
    tma_load_2d(tile_s, &tm_in, x, y, bar_s);
  }
  load_twiddles(s_tw, p.W256);
  if (threadIdx.x == 0) {
    // bounded wait (about a second): the copy of 32 KB takes microseconds
    int ok = 0;
    for (int it = 0; it < (1 << 22); it++)
      if (mbar_try_wait(bar_s, 0)) {
        ok = 1;
        break;
      }
    s_ok = ok;
    if (!ok) {
      atomicCAS(const_cast<int32_t*>(&p.ctrl->err), 0, (int32_t)WP_ETIMEOUT);
      // let a late copy land before the block's shared memory is given up (bounded too)
      for (int it = 0; it < (1 << 22) && !mbar_try_wait(bar_s, 0); it++) {
      }
    }
  }
  __syncthreads();
  if (!s_ok) return;
  (void)mbar_try_wait(bar_s, 0);  // the completed phase: acquire the copy for this thread

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 4, t = lane & 15;
  const int l = 2 * warp + g;
  cx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = *reinterpret_cast<const cx<float>*>(tile + swz(t + 16 * r, l));
  __syncthreads();  // every line is in registers: the region now holds the transposes
  cx<float>* reg = reinterpret_cast<cx<float>*>(tile) + l * kLS;
  if constexpr (KIN) {
    const TwE<float> L = p.lines_kin[cb + l].L;
    kinetic256(p, v, reg, s_tw, L, t);
  } else if (p.flags & F_IFFT) {
    fft256<true>(v, reg, s_tw, t);
  } else {
    fft256<false>(v, reg, s_tw, t);
  }
  [[maybe_unused]] float qs[8];
  if constexpr (OBS) {
#pragma unroll
    for (int j = 0; j < 8; j++) qs[j] = 0.0f;
    mom_sums256(p, v, t, qs);
    if (p.flags & F_NO_STORE) {
      obs256_partials(p, qs, o, cb + l, l, t);
      return;
    }
  }
  __syncthreads();  // every transpose is done: back to the swizzled tile layout
#pragma unroll
  for (int r = 0; r < 16; r++) *reinterpret_cast<cx<float>*>(tile + swz(t + 16 * r, l)) = v[r];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) tma_store_2d(&tm_out, x, y, tile_s);
  if constexpr (OBS) obs256_partials(p, qs, o, cb + l, l, t);
}

}  // namespace p256
}  // namespace wp
