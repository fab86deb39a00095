// complex128 (FP64) instantiation of the split-operator kernels, plus the
// precision-independent kernels.
#define WP_COMMON_KERNELS 1
#include "wp_launch.cuh"

namespace wp {

WP_INSTANTIATE(double)

int launch_reduce(const ReduceParams& p, void* stream) {
  k_reduce<<<1, 256, 0, (cudaStream_t)stream>>>(p);
  return cuda_status(cudaGetLastError());
}

int launch_set_step(Ctrl* ctrl, int64_t step, void* stream) {
  k_set_step<<<1, 1, 0, (cudaStream_t)stream>>>(ctrl, step);
  return cuda_status(cudaGetLastError());
}

int launch_add_step(Ctrl* ctrl, int64_t add, void* stream) {
  k_add_step<<<1, 1, 0, (cudaStream_t)stream>>>(ctrl, add);
  return cuda_status(cudaGetLastError());
}

}  // namespace wp
