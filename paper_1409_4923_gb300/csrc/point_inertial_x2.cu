// point_inertial_x2.cu -- instantiations of the single-point path kernel for model 0 (inertial washboard),
// 2 paths per lane.
#include "point_kernels.cuh"

namespace sde {

SDE_POINT_UNIT(0, 2)

}  // namespace sde
