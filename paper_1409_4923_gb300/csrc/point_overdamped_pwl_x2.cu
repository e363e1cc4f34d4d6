// point_overdamped_pwl_x2.cu -- instantiations of the single-point path kernel for model 2 (overdamped piecewise-linear),
// 2 paths per lane.
#include "point_kernels.cuh"

namespace sde {

SDE_POINT_UNIT(2, 2)

}  // namespace sde
