// Batched contiguous-axis pass kernel (potential phase) for the complex64 form.
#include "wp_batch_launch.cuh"

WP_BATCH_TU(float, true, launch_pass_batch_contig)
