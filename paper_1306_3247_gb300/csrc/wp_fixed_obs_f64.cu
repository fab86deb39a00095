// Fixed-size pass kernels with the observable partial sums for the complex128 (FP64) form.
#include "wp_fixed_launch.cuh"

WP_FIXED_TU(double, true, false, launch_fixed_obs, fixed_obs_smem_limit_set)
