// Fixed-size pass kernels with the observable partial sums for the complex64 form.
#include "wp_fixed_launch.cuh"

WP_FIXED_TU(float, true, false, launch_fixed_obs, fixed_obs_smem_limit_set)
