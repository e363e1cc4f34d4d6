// point_overdamped_pwl.cu -- instantiations of the single-point path kernel for model 2.
#include "point_kernels.cuh"

namespace sde {

cudaError_t launch_point_m2(bool pois, bool dich, int gauss, const PointConsts& P,
                              const LaunchConsts& K, const Workspace& ws, const PathOutPtrs& po,
                              int bt, int gb, int sm, cudaStream_t st)
{
    return launch_point_model<2>(pois, dich, gauss, P, K, ws, po, bt, gb, sm, st);
}

int blocks_per_sm_m2(bool pois, bool dich, int gauss, int bt)
{
    return blocks_per_sm_model<2>(pois, dich, gauss, bt);
}

}  // namespace sde
