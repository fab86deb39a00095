// Fixed-size pass kernels without partial sums for the complex64 form.
#include "wp_fixed_launch.cuh"

WP_FIXED_TU(float, false, false, launch_fixed, fixed_smem_limit_set)
