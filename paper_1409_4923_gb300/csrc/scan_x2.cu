// scan_x2.cu -- the batched scan with two paths per lane on packed FP32 pairs.
//
// Sec. 5 runs many parameter values in one kernel call.  Here each work item
// is 64 paths of one point (its 32-path tiles 2k and 2k + 1); a lane
// integrates paths first + lane and first + 32 + lane with chunk_steps_x2,
// the point's constants read from the point table in global memory, and the
// dichotomous flips drawn a window ahead in shared memory.  Each 32-path tile
// writes its own FP64 partial record, so a point's records and their fold are
// those of its single-point run, bit for bit.  Without Poisson noise only:
// the Poissonian variants keep one path per lane (scan_kernel).
#include "launch.h"

namespace sde {

template <int DICH, int GAUSS>
__global__ void __launch_bounds__(128, 6) scan_kernel_x2(const PointConsts* __restrict__ pts,
                                                      const uint2* __restrict__ items,
                                                      const __grid_constant__ LaunchConsts K,
                                                      uint32_t* __restrict__ counter,
                                                      int32_t* __restrict__ status,
                                                      double* __restrict__ partials)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t t0 = K.budget_ns ? globaltimer_ns() : 0ull;
    uint32_t* win = nullptr;
    if constexpr (WindowedFlips<kModelInertial, false, DICH, GAUSS, 2>::value) {
        extern __shared__ uint32_t sde_scan_smem[];
        win = sde_scan_smem + (threadIdx.x >> 5) * kWinWordsPerWarp;
    }
    for (;;) {
        const uint32_t item = next_item(counter, status, K, lane, t0);
        if (item == 0xffffffffu) break;
        const uint2 it = items[item];
        const PointConsts& P = pts[it.x];
        const uint32_t path[2] = {it.y + lane, it.y + 32u + lane};
        PathResult R[2];
        simulate_paths<kModelInertial, false, DICH, GAUSS, 2>(P, K, path, lane, R, win);
        store_partial(partials, 2u * item, lane, path[0] < P.n_paths, R[0]);
        store_partial(partials, 2u * item + 1u, lane, path[1] < P.n_paths, R[1]);
    }
}

template <int DICH, int GAUSS>
static cudaError_t launch_scan_x2_t(const PointConsts* pts, const uint2* items, const LaunchConsts& K,
                                    const Workspace& ws, int bt, int gb, int sm, cudaStream_t st)
{
    auto kern = scan_kernel_x2<DICH, GAUSS>;
    const size_t smem = WindowedFlips<kModelInertial, false, DICH, GAUSS, 2>::value
                            ? (size_t)(bt / 32) * kWinWordsPerWarp * sizeof(uint32_t) : 0u;
    if (gb <= 0) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, bt, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        const uint64_t need = ((uint64_t)K.n_items * 32ull + bt - 1) / bt;
        const uint64_t cap = (uint64_t)per_sm * (uint64_t)sm;
        gb = (int)(need < cap ? need : cap);
        if (gb < 1) gb = 1;
    }
    kern<<<gb, bt, smem, st>>>(pts, items, K, ws.counter, ws.status, ws.partials);
    return cudaGetLastError();
}

cudaError_t launch_scan_x2(int dich, int gauss, const PointConsts* pts, const uint2* items,
                           const LaunchConsts& K, const Workspace& ws, int bt, int gb, int sm,
                           cudaStream_t st)
{
#define SDE_SCAN2(DI, GA) \
    if (dich == DI && gauss == GA) return launch_scan_x2_t<DI, GA>(pts, items, K, ws, bt, gb, sm, st);
    SDE_SCAN2(1, kGauss3Point) SDE_SCAN2(0, kGauss3Point) SDE_SCAN2(2, kGauss3Point)
    SDE_SCAN2(1, 0) SDE_SCAN2(0, 0) SDE_SCAN2(2, 0)
#undef SDE_SCAN2
    return cudaErrorInvalidValue;
}

}  // namespace sde
