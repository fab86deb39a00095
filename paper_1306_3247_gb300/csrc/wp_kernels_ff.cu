// Complex128-accuracy form computed in float-float (FP32 pair) arithmetic.
#include "wp_launch.cuh"

namespace wp {

WP_INSTANTIATE(ff)

}  // namespace wp
