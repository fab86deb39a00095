// Batched contiguous-axis pass kernel (potential phase) for the complex128 (FP64) form.
#include "wp_batch_launch.cuh"

WP_BATCH_TU(double, true, launch_pass_batch_contig)
