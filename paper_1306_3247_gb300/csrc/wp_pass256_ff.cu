// Two-stage 256-point pass kernels of the float-float complex128-accuracy form.
#include "wp_pass256_launch.cuh"

WP_PASS256_TU(ff)
