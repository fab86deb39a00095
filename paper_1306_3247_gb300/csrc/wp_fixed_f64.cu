// Fixed-size pass kernels without partial sums for the complex128 (FP64) form.
#include "wp_fixed_launch.cuh"

WP_FIXED_TU(double, false, false, launch_fixed, fixed_smem_limit_set)
