// One-launch-per-pass batched kernel: float, kinetic (strided) pass.
#include "wp_batch_merged.cuh"

WP_MERGED_TU(float, false, launch_merged_strided)
