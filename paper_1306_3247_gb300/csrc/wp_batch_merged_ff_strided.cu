// One-launch-per-pass batched kernel: ff, kinetic (strided) pass.
#include "wp_batch_merged.cuh"

WP_MERGED_TU(ff, false, launch_merged_strided)
