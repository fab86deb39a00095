// Batched strided-axis pass kernel (kinetic factor) for the complex128 (FP64) form.
#include "wp_batch_launch.cuh"

WP_BATCH_TU(double, false, launch_pass_batch_strided)
