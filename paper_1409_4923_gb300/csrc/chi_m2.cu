// chi_m2.cu -- instantiations of the local-error diagnostic kernel for model 2.
#include "chi_kernels.cuh"

namespace sde {

cudaError_t launch_chi_m2(bool pois, int dich, int gauss, const PointConsts& P, const LaunchConsts& K,
                          uint32_t n_steps, const Workspace& ws, int bt, int gb, int sm, cudaStream_t st)
{
    return launch_chi_model<2>(pois, dich, gauss, P, K, n_steps, ws, bt, gb, sm, st);
}

}  // namespace sde
