// complex64 (FP32 FFT, FP64 tables and reductions) instantiation of the kernels.
#include "wp_launch.cuh"

namespace wp {

WP_INSTANTIATE(float)

}  // namespace wp
