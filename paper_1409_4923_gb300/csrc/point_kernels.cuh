// point_kernels.cuh -- the single-point path kernel and its instantiation table.
#pragma once
#include "launch.h"

namespace sde {

// Persistent warp-item loop for one parameter point: each warp pulls 32-path
// items (PPT consecutive items at a time, one path of each per lane),
// integrates its lanes' paths for n_transient + n_avg steps and writes each
// item's FP64 partial sums (and, optionally, per-path results).
template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
__device__ __forceinline__ void point_items(const PointConsts& P, const LaunchConsts& K,
                                            uint32_t* __restrict__ counter, int32_t* __restrict__ status,
                                            double* __restrict__ partials, const PathOutPtrs& po)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t t0 = K.budget_ns ? globaltimer_ns() : 0ull;
    uint32_t* win = nullptr;
    if constexpr (WindowedFlips<MODEL, POIS, DICH, GAUSS, PPT>::value) {
        extern __shared__ uint32_t sde_point_smem[];
        win = sde_point_smem + (threadIdx.x >> 5) * kWinWordsPerWarp;
    }
    constexpr bool kKickWin = PPT == 1 && WindowedKicks<POIS, GAUSS>::value;
    if constexpr (kKickWin) {
        extern __shared__ uint32_t sde_point_smem[];
        win = sde_point_smem + (threadIdx.x >> 5) * kKickWordsPerWarp + lane;
    }
    if constexpr (WindowedKicks2<MODEL, POIS, DICH, GAUSS, PPT>::value) {
        extern __shared__ uint32_t sde_point_smem[];
        win = sde_point_smem + (threadIdx.x >> 5) * kKick2WordsPerWarp;
    }
    for (;;) {
        const uint32_t item = next_item(counter, status, K, lane, t0, (uint32_t)PPT);
        if (item == 0xffffffffu) break;
        // local: the path's index within the run (outputs); path0 + local:
        // its index in the random counter
        if (PPT == 1) {
            const uint32_t local = item * 32u + lane;
            const bool valid = local < P.n_paths;
            PathResult R;
            simulate_path<MODEL, POIS, DICH, GAUSS, kKickWin>(P, K, P.path0 + local, lane, R, win);
            if (valid) store_path(po, local, R);
            store_partial(partials, item, lane, valid, R);
        } else {
            uint32_t path[PPT];
#pragma unroll
            for (int p = 0; p < PPT; ++p) path[p] = P.path0 + (item + (uint32_t)p) * 32u + lane;
            PathResult R[PPT];
            simulate_paths<MODEL, POIS, DICH, GAUSS, PPT>(P, K, path, lane, R, win);
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                if (item + (uint32_t)p >= K.n_items) break;      // past the last item: no output
                const uint32_t local = (item + (uint32_t)p) * 32u + lane;
                const bool valid = local < P.n_paths;
                if (valid) store_path(po, local, R[p]);
                store_partial(partials, item + (uint32_t)p, lane, valid, R[p]);
            }
        }
    }
}

template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
__global__ void __launch_bounds__(128) point_kernel(const __grid_constant__ PointConsts P,
                                                    const __grid_constant__ LaunchConsts K,
                                                    uint32_t* __restrict__ counter,
                                                    int32_t* __restrict__ status,
                                                    double* __restrict__ partials,
                                                    const PathOutPtrs po)
{
    point_items<MODEL, POIS, DICH, GAUSS, PPT>(P, K, counter, status, partials, po);
}

// The same loop compiled for six resident blocks of 128 threads (at most 80
// registers, 24 warps per SM).  Two paths per lane run here: without Poisson
// noise (measured on the 2^20-path dichotomous run before the flip windows,
// 573 ms against 583 ms at 96 registers (five blocks), 576 ms at 72 and
// 592 ms at 64, where the spills reach the step loop; uncapped, 123
// registers and 16 warps, 599 ms), and with Poisson noise in kick windows.
template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
__global__ void __launch_bounds__(128, 6) point_kernel_capped(const __grid_constant__ PointConsts P,
                                                              const __grid_constant__ LaunchConsts K,
                                                              uint32_t* __restrict__ counter,
                                                              int32_t* __restrict__ status,
                                                              double* __restrict__ partials,
                                                              const PathOutPtrs po)
{
    point_items<MODEL, POIS, DICH, GAUSS, PPT>(P, K, counter, status, partials, po);
}

template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
constexpr auto point_kernel_for()
{
    if constexpr (PPT == 2 && (!POIS || WindowedKicks2<MODEL, POIS, DICH, GAUSS, PPT>::value))
        return point_kernel_capped<MODEL, POIS, DICH, GAUSS, PPT>;
    else return point_kernel<MODEL, POIS, DICH, GAUSS, PPT>;
}

// Dynamic shared memory of a launch: the flip or kick windows of its warps.
template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
constexpr size_t point_smem_bytes(int block_threads)
{
    if (WindowedFlips<MODEL, POIS, DICH, GAUSS, PPT>::value)
        return (size_t)(block_threads / 32) * kWinWordsPerWarp * sizeof(uint32_t);
    if (PPT == 1 && WindowedKicks<POIS, GAUSS>::value)
        return (size_t)(block_threads / 32) * kKickWordsPerWarp * sizeof(uint32_t);
    if (WindowedKicks2<MODEL, POIS, DICH, GAUSS, PPT>::value)
        return (size_t)(block_threads / 32) * kKick2WordsPerWarp * sizeof(uint32_t);
    return 0u;
}

template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
cudaError_t launch_point_t(const PointConsts& P, const LaunchConsts& K, const Workspace& ws,
                           const PathOutPtrs& po, int block_threads, int grid_blocks,
                           int sm_count, cudaStream_t st)
{
    auto kern = point_kernel_for<MODEL, POIS, DICH, GAUSS, PPT>();
    const size_t smem = point_smem_bytes<MODEL, POIS, DICH, GAUSS, PPT>(block_threads);
    if (grid_blocks <= 0) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block_threads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        const uint64_t warps = ((uint64_t)K.n_items + PPT - 1) / PPT;
        const uint64_t need = (warps * 32ull + block_threads - 1) / block_threads;
        uint64_t cap = (uint64_t)per_sm * (uint64_t)sm_count;
        grid_blocks = (int)(need < cap ? need : cap);
        if (grid_blocks < 1) grid_blocks = 1;
    }
    kern<<<grid_blocks, block_threads, smem, st>>>(P, K, ws.counter, ws.status, ws.partials, po);
    return cudaGetLastError();
}

template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
int blocks_per_sm_t(int block_threads)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, point_kernel_for<MODEL, POIS, DICH, GAUSS, PPT>(),
                                                  block_threads,
                                                  point_smem_bytes<MODEL, POIS, DICH, GAUSS, PPT>(block_threads));
    return per_sm;
}

// Dispatch over the noise switches for one model and paths-per-lane count
// (each pair instantiated in its own translation unit).
template <int MODEL, int PPT>
cudaError_t launch_point_model(bool pois, int dich, int gauss, const PointConsts& P,
                               const LaunchConsts& K, const Workspace& ws, const PathOutPtrs& po,
                               int bt, int gb, int sm, cudaStream_t st)
{
#define SDE_CASE(PO, DI, GA) \
    if (pois == PO && dich == DI && gauss == GA) \
        return launch_point_t<MODEL, PO, DI, GA, PPT>(P, K, ws, po, bt, gb, sm, st);
    SDE_FOR_EACH_VARIANT(SDE_CASE)
#undef SDE_CASE
    return cudaErrorInvalidValue;
}

template <int MODEL, int PPT>
int blocks_per_sm_model(bool pois, int dich, int gauss, int bt)
{
#define SDE_CASE(PO, DI, GA) \
    if (pois == PO && dich == DI && gauss == GA) return blocks_per_sm_t<MODEL, PO, DI, GA, PPT>(bt);
    SDE_FOR_EACH_VARIANT(SDE_CASE)
#undef SDE_CASE
    return 0;
}

// Instantiation unit of one (model, paths per lane) pair.
#define SDE_POINT_UNIT(M, PPT) \
    cudaError_t launch_point_m##M##_p##PPT(bool pois, int dich, int gauss, const PointConsts& P, \
                                          const LaunchConsts& K, const Workspace& ws, \
                                          const PathOutPtrs& po, int bt, int gb, int sm, cudaStream_t st) \
    { \
        return launch_point_model<M, PPT>(pois, dich, gauss, P, K, ws, po, bt, gb, sm, st); \
    } \
    int blocks_per_sm_m##M##_p##PPT(bool pois, int dich, int gauss, int bt) \
    { \
        return blocks_per_sm_model<M, PPT>(pois, dich, gauss, bt); \
    }

}  // namespace sde
