// Fixed-size pass kernels with the observable partial sums for the float-float complex128-accuracy form.
#include "wp_fixed_launch.cuh"

WP_FIXED_TU(ff, true, false, launch_fixed_obs, fixed_obs_smem_limit_set)
