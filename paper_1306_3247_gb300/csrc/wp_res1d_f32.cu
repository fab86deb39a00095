// Fixed-length resident-line kernels (1-D propagation) for the complex64 form.
#include <type_traits>

#include "wp_res1d_launch.cuh"

WP_RES1D_TU(float)
