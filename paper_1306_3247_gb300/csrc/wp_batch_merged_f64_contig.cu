// One-launch-per-pass batched kernel: double, potential (contiguous) pass.
#include "wp_batch_merged.cuh"

WP_MERGED_TU(double, true, launch_merged_contig)
