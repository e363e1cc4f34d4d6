// point_inertial.cu -- instantiations of the single-point path kernel for model 0 (inertial washboard),
// 1 path per lane.
#include "point_kernels.cuh"

namespace sde {

SDE_POINT_UNIT(0, 1)

}  // namespace sde
