// One-launch-per-pass batched kernel: ff, potential (contiguous) pass.
#include "wp_batch_merged.cuh"

WP_MERGED_TU(ff, true, launch_merged_contig)
