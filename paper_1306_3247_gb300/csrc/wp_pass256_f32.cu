// Two-stage 256-point pass kernels of the complex64 form.
#include "wp_pass256_launch.cuh"

WP_PASS256_TU(float)
