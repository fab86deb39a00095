// One-launch-per-pass batched kernel: float, potential (contiguous) pass.
#include "wp_batch_merged.cuh"

WP_MERGED_TU(float, true, launch_merged_contig)
