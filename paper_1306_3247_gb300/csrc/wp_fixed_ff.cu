// Fixed-size pass kernels without partial sums for the float-float complex128-accuracy form.
#include "wp_fixed_launch.cuh"

WP_FIXED_TU(ff, false, false, launch_fixed, fixed_smem_limit_set)
