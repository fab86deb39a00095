// complex128 (FP64) instantiation of the split-operator kernels, plus the
// precision-independent kernels.
#define WP_COMMON_KERNELS 1
#include "wp_launch.cuh"

namespace wp {

WP_INSTANTIATE(double)

int launch_reduce_rows(ReduceParams& p, void* stream) {
  const int64_t rows = p.npos > p.nmom ? p.npos : p.nmom;
  if (rows <= 512) return 0;
  // runs of at least 256 rows, at most about two blocks per SM
  int64_t R = (rows + 303) / 304;
  if (R < 256) R = 256;
  const unsigned nb = (unsigned)((rows + R - 1) / R);
  k_reduce_rows<<<dim3(nb, 2), 256, 0, (cudaStream_t)stream>>>(const_cast<double*>(p.pos), p.npos,
                                                                 const_cast<double*>(p.mom), p.nmom, R);
  p.npos = (p.npos + R - 1) / R;
  p.nmom = (p.nmom + R - 1) / R;
  p.pos_stride = p.mom_stride = R;
  return cuda_status(cudaGetLastError());
}

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
