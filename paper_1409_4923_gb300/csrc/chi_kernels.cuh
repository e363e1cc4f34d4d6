// chi_kernels.cuh -- the local-error diagnostic kernel and its instantiation table.
#pragma once
#include "launch.h"

namespace sde {

__device__ __forceinline__ float warp_max_nonneg(float x)
{
    // non-negative floats order like their bit patterns
    return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(x)));
}

// Sec. 4's chi = predictor - corrector (without the jump increments) over
// steps [0, n_steps) of every path from its initial state, one step at a
// time with the engine's own step code.  Each 32-path item writes {paths,
// sum chi_x^2, sum chi_v^2, max |chi_x|, max |chi_v|} (coordinate units for
// chi_x); the host folds the items.  The FP32 squares are moved to FP64
// every 256 steps.
template <int MODEL, bool POIS, int DICH, int GAUSS>
__global__ void __launch_bounds__(128) chi_kernel(const __grid_constant__ PointConsts P,
                                                  const __grid_constant__ LaunchConsts K, uint32_t n_steps,
                                                  uint32_t* __restrict__ counter, int32_t* __restrict__ status,
                                                  double* __restrict__ partials)
{
    const uint32_t lane = threadIdx.x & 31u;
    for (;;) {
        const uint32_t item = next_item(counter, status, K, lane, 0ull);
        if (item == 0xffffffffu) break;
        const uint32_t path = item * 32u + lane;
        PathState S;
        init_path<MODEL, POIS, DICH>(S, P, K, path);
        double sx = 0.0, sv = 0.0;
        float ax = 0.0f, av = 0.0f, mx = 0.0f, mv = 0.0f;
        for (uint32_t n = 0; n < n_steps; ++n) {
            const float dxi = gauss_at<GAUSS>(P, K, path, n);
            float pj, dg;
            jumps_inline<POIS, DICH>(S, P, K, path, n, pj, dg);
            float chi[2];
            pc_step<MODEL, POIS, DICH, false, true, true>(S, P, dxi, pj, dg, drive_at(n, P), drive_at(n + 1u, P),
                                                          chi);
            ax = fmaf(chi[0], chi[0], ax);
            av = fmaf(chi[1], chi[1], av);
            mx = fmaxf(mx, fabsf(chi[0]));
            mv = fmaxf(mv, fabsf(chi[1]));
            if ((n & 255u) == 255u) {
                sx += (double)ax;
                sv += (double)av;
                ax = av = 0.0f;
            }
        }
        sx += (double)ax;
        sv += (double)av;
        const bool valid = path < P.n_paths;
        const double cnt = warp_sum(valid ? 1.0 : 0.0);
        sx = warp_sum(valid ? sx : 0.0);
        sv = warp_sum(valid ? sv : 0.0);
        mx = warp_max_nonneg(valid ? mx : 0.0f);
        mv = warp_max_nonneg(valid ? mv : 0.0f);
        if (lane == 0u) {
            double* o = partials + 5ull * item;
            o[0] = cnt; o[1] = sx; o[2] = sv; o[3] = (double)mx; o[4] = (double)mv;
        }
    }
}

template <int MODEL, bool POIS, int DICH, int GAUSS>
cudaError_t launch_chi_t(const PointConsts& P, const LaunchConsts& K, uint32_t n_steps, const Workspace& ws,
                         int block_threads, int grid_blocks, int sm_count, cudaStream_t st)
{
    auto kern = chi_kernel<MODEL, POIS, DICH, GAUSS>;
    if (grid_blocks <= 0) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block_threads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        const uint64_t need = ((uint64_t)K.n_items * 32ull + block_threads - 1) / block_threads;
        const uint64_t cap = (uint64_t)per_sm * (uint64_t)sm_count;
        grid_blocks = (int)(need < cap ? need : cap);
        if (grid_blocks < 1) grid_blocks = 1;
    }
    kern<<<grid_blocks, block_threads, 0, st>>>(P, K, n_steps, ws.counter, ws.status, ws.partials);
    return cudaGetLastError();
}

template <int MODEL>
cudaError_t launch_chi_model(bool pois, int dich, int gauss, const PointConsts& P, const LaunchConsts& K,
                             uint32_t n_steps, const Workspace& ws, int bt, int gb, int sm, cudaStream_t st)
{
#define SDE_CASE(PO, DI, GA) \
    if (pois == PO && dich == DI && gauss == GA) \
        return launch_chi_t<MODEL, PO, DI, GA>(P, K, n_steps, ws, bt, gb, sm, st);
    SDE_FOR_EACH_VARIANT(SDE_CASE)
#undef SDE_CASE
    return cudaErrorInvalidValue;
}

}  // namespace sde
