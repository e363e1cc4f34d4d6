// point_overdamped_pwl.cu -- instantiations of the single-point path kernel for model 2 (overdamped piecewise-linear),
// 1 path per lane.
#include "point_kernels.cuh"

namespace sde {

SDE_POINT_UNIT(2, 1)

}  // namespace sde
