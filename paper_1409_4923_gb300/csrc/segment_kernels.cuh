// segment_kernels.cuh -- the segmented-run path kernel and its instantiation table.
#pragma once
#include "launch.h"

namespace sde {

// One segment of a segmented run (Algorithm 5): each warp pulls 32-path
// items, loads its lane's path state (or draws it when na == 0), advances it
// over steps [na, nb) and saves it.  The segment that ends the run also
// writes the item's FP64 partial sums (and, optionally, per-path results), so
// the fold that follows gives the statistics of sde_run.
template <int MODEL, bool POIS, int DICH, int GAUSS>
__global__ void __launch_bounds__(128) segment_kernel(const __grid_constant__ PointConsts P,
                                                      const __grid_constant__ LaunchConsts K,
                                                      const StatePlanes M, uint32_t na, uint32_t nb,
                                                      uint32_t* __restrict__ counter,
                                                      int32_t* __restrict__ status,
                                                      double* __restrict__ partials,
                                                      const PathOutPtrs po)
{
    const uint32_t lane = threadIdx.x & 31u;
    const bool last = nb == P.n_tr + P.n_avg;
    for (;;) {
        const uint32_t item = next_item(counter, status, K, lane, 0ull);
        if (item == 0xffffffffu) break;
        const uint32_t local = item * 32u + lane;       // state plane and output index
        const uint32_t path = P.path0 + local;           // random-counter index
        PathState S;
        if (na == 0u) init_path<MODEL, POIS, DICH>(S, P, K, path);
        else load_state(S, M, local);
        advance_path<MODEL, POIS, DICH, GAUSS>(S, P, K, path, lane, na, nb);
        store_state(S, M, local);
        if (last) {
            const bool valid = local < P.n_paths;
            PathResult R;
            finish_path<MODEL, POIS, DICH>(S, P, R);
            if (valid) store_path(po, local, R);
            store_partial(partials, item, lane, valid, R);
        }
    }
}

template <int MODEL, bool POIS, int DICH, int GAUSS>
cudaError_t launch_segment_t(const PointConsts& P, const LaunchConsts& K, const StatePlanes& M,
                             uint32_t na, uint32_t nb, const Workspace& ws, const PathOutPtrs& po,
                             int block_threads, int grid_blocks, int sm_count, cudaStream_t st)
{
    auto kern = segment_kernel<MODEL, POIS, DICH, GAUSS>;
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
    kern<<<grid_blocks, block_threads, 0, st>>>(P, K, M, na, nb, ws.counter, ws.status, ws.partials, po);
    return cudaGetLastError();
}

template <int MODEL>
cudaError_t launch_segment_model(bool pois, int dich, int gauss, const PointConsts& P,
                                 const LaunchConsts& K, const StatePlanes& M, uint32_t na,
                                 uint32_t nb, const Workspace& ws, const PathOutPtrs& po, int bt,
                                 int gb, int sm, cudaStream_t st)
{
#define SDE_CASE(PO, DI, GA) \
    if (pois == PO && dich == DI && gauss == GA) \
        return launch_segment_t<MODEL, PO, DI, GA>(P, K, M, na, nb, ws, po, bt, gb, sm, st);
    SDE_FOR_EACH_VARIANT(SDE_CASE)
#undef SDE_CASE
    return cudaErrorInvalidValue;
}

}  // namespace sde
