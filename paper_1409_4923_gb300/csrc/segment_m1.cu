// segment_m1.cu -- instantiations of the segmented-run path kernel for model 1.
#include "segment_kernels.cuh"

namespace sde {

cudaError_t launch_segment_m1(bool pois, int dich, int gauss, const PointConsts& P,
                              const LaunchConsts& K, const StatePlanes& M, uint32_t na, uint32_t nb,
                              const Workspace& ws, const PathOutPtrs& po, int bt, int gb, int sm,
                              cudaStream_t st)
{
    return launch_segment_model<1>(pois, dich, gauss, P, K, M, na, nb, ws, po, bt, gb, sm, st);
}

}  // namespace sde
