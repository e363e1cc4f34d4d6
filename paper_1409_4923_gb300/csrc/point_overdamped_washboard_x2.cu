// point_overdamped_washboard_x2.cu -- instantiations of the single-point path kernel for model 1 (overdamped washboard),
// 2 paths per lane.
#include "point_kernels.cuh"

namespace sde {

SDE_POINT_UNIT(1, 2)

}  // namespace sde
