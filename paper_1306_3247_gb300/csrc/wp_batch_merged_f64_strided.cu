// One-launch-per-pass batched kernel: double, kinetic (strided) pass.
#include "wp_batch_merged.cuh"

WP_MERGED_TU(double, false, launch_merged_strided)
