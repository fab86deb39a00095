// Batched strided-axis pass kernel (kinetic factor) for the float-float complex128-accuracy form.
#include "wp_batch_launch.cuh"

WP_BATCH_TU(ff, false, launch_pass_batch_strided)
