// point_overdamped_washboard.cu -- instantiations of the single-point path kernel for model 1 (overdamped washboard),
// 1 path per lane.
#include "point_kernels.cuh"

namespace sde {

SDE_POINT_UNIT(1, 1)

}  // namespace sde
