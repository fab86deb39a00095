// Batched strided-axis pass kernel (kinetic factor) for the complex64 form.
#include "wp_batch_launch.cuh"

WP_BATCH_TU(float, false, launch_pass_batch_strided)
