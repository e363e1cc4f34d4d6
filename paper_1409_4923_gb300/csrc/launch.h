// launch.h -- host-side launchers of the engine's kernels (internal header).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "engine.cuh"

namespace sde {

// Every kernel variant: X(poisson, dichotomous kind, gauss kind) with the
// dichotomous kind 0 (off), 1 (corrector increment, Algorithm 1) or 2 (part
// of the drift), and the Gaussian kind 0 (off), three-point or Box-Muller.
#define SDE_FOR_EACH_VARIANT(X) \
    X(false, 0, 0) X(true, 0, 0) X(false, 1, 0) X(true, 1, 0) X(false, 2, 0) X(true, 2, 0) \
    X(false, 0, kGauss3Point) X(true, 0, kGauss3Point) X(false, 1, kGauss3Point) \
    X(true, 1, kGauss3Point) X(false, 2, kGauss3Point) X(true, 2, kGauss3Point) \
    X(false, 0, kGaussNormal) X(true, 0, kGaussNormal) X(false, 1, kGaussNormal) \
    X(true, 1, kGaussNormal) X(false, 2, kGaussNormal) X(true, 2, kGaussNormal)

struct Workspace {
    uint32_t* counter;   // work-item counter (must start at 0)
    int32_t* status;     // kStatusOk / kStatusTimedOut (must start at 0)
    double* partials;    // 5 doubles per warp item
};

// Launch the single-point path kernel for (model, poisson, dichotomous, gauss)
// with ppt (1 or 2) paths per lane.  grid_blocks == 0 picks a persistent grid
// from the occupancy calculator.
cudaError_t launch_point(int model, bool pois, int dich, int gauss, int ppt, const PointConsts& P,
                         const LaunchConsts& K, const Workspace& ws, const PathOutPtrs& po,
                         int block_threads, int grid_blocks, int sm_count, cudaStream_t st);

// One segment [na, nb) of a segmented run over the saved path states M
// (na == 0 draws the initial states; nb == n_transient + n_avg also writes
// the item partials and per-path results).
cudaError_t launch_segment(int model, bool pois, int dich, int gauss, const PointConsts& P,
                           const LaunchConsts& K, const StatePlanes& M, uint32_t na, uint32_t nb,
                           const Workspace& ws, const PathOutPtrs& po, int block_threads,
                           int grid_blocks, int sm_count, cudaStream_t st);

// Sec. 4's local-error indicator over steps [0, n_steps) of every path:
// item partials {paths, sum chi_x^2, sum chi_v^2, max |chi_x|, max |chi_v|}.
cudaError_t launch_chi(int model, bool pois, int dich, int gauss, const PointConsts& P,
                       const LaunchConsts& K, uint32_t n_steps, const Workspace& ws, int block_threads,
                       int grid_blocks, int sm_count, cudaStream_t st);

// Inertial-washboard scan kernel over an item table of (point, first path);
// gauss is 0 (no Gaussian noise) or the three-point law.
cudaError_t launch_scan(bool pois, int dich, int gauss, const PointConsts* pts_dev,
                        const uint2* items_dev,
                        const LaunchConsts& K, const Workspace& ws, int block_threads,
                        int grid_blocks, int sm_count, cudaStream_t st);

// The same scan without Poisson noise, two paths per lane: item k is 64 paths
// (point, first path) and writes the partial records 2k and 2k + 1 of its two
// 32-path tiles.
cudaError_t launch_scan_x2(int dich, int gauss, const PointConsts* pts_dev, const uint2* items_dev,
                           const LaunchConsts& K, const Workspace& ws, int block_threads,
                           int grid_blocks, int sm_count, cudaStream_t st);

// Fixed-order FP64 fold of item partials: ranges[p] = (first item, item count),
// out5[5 p .. 5 p + 4] receives the point's five sums.
cudaError_t launch_fold(const double* partials, const uint2* ranges, uint32_t npts,
                        double* out5, cudaStream_t st);

// Warp items of 32 doubles -> partials {n, sum, sum of squares, 0, 0}.
cudaError_t launch_reduce_items(const double* vals, uint64_t n, double* partials, cudaStream_t st);

cudaError_t launch_philox(const uint4* ctr, uint64_t n, const LaunchConsts& K, uint4* out,
                          cudaStream_t st);

// Occupancy-derived resident blocks per SM for the kernel a launch would use.
int point_blocks_per_sm(int model, bool pois, int dich, int gauss, int ppt, int block_threads);

}  // namespace sde
