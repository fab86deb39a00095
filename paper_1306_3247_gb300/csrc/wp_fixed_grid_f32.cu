// Fixed-size contiguous pass kernels with a static grid potential (without and with the
// observable partial sums) for the complex64 form.
#include "wp_fixed_launch.cuh"

WP_FIXED_TU(float, false, true, launch_fixed_grid, fixed_grid_smem_limit_set)
WP_FIXED_TU(float, true, true, launch_fixed_grid_obs, fixed_grid_obs_smem_limit_set)
