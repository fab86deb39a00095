// Batched contiguous-axis pass kernel (potential phase) for the float-float complex128-accuracy form.
#include "wp_batch_launch.cuh"

WP_BATCH_TU(ff, true, launch_pass_batch_contig)
