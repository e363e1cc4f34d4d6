// aux_kernels.cu -- batched-scan kernel, deterministic FP64 fold, reduction
// and Philox test kernels, and the launcher table.
#include "launch.h"

namespace sde {

#define SDE_POINT_DECL(M, PPT) \
cudaError_t launch_point_m##M##_p##PPT(bool, int, int, const PointConsts&, const LaunchConsts&, \
                                      const Workspace&, const PathOutPtrs&, int, int, int, cudaStream_t); \
int blocks_per_sm_m##M##_p##PPT(bool, int, int, int);
SDE_POINT_DECL(0, 1) SDE_POINT_DECL(1, 1) SDE_POINT_DECL(2, 1)
SDE_POINT_DECL(0, 2) SDE_POINT_DECL(1, 2) SDE_POINT_DECL(2, 2)
#undef SDE_POINT_DECL
#define SDE_SEG_DECL(M) \
cudaError_t launch_segment_m##M(bool, int, int, const PointConsts&, const LaunchConsts&, \
                                const StatePlanes&, uint32_t, uint32_t, const Workspace&, \
                                const PathOutPtrs&, int, int, int, cudaStream_t);
SDE_SEG_DECL(0) SDE_SEG_DECL(1) SDE_SEG_DECL(2)
#undef SDE_SEG_DECL
#define SDE_CHI_DECL(M) \
cudaError_t launch_chi_m##M(bool, int, int, const PointConsts&, const LaunchConsts&, uint32_t, \
                            const Workspace&, int, int, int, cudaStream_t);
SDE_CHI_DECL(0) SDE_CHI_DECL(1) SDE_CHI_DECL(2)
#undef SDE_CHI_DECL

cudaError_t launch_chi(int model, bool pois, int dich, int gauss, const PointConsts& P,
                       const LaunchConsts& K, uint32_t n_steps, const Workspace& ws, int bt, int gb, int sm,
                       cudaStream_t st)
{
    switch (model) {
    case kModelInertial: return launch_chi_m0(pois, dich, gauss, P, K, n_steps, ws, bt, gb, sm, st);
    case kModelOverdampedWashboard: return launch_chi_m1(pois, dich, gauss, P, K, n_steps, ws, bt, gb, sm, st);
    case kModelPWL: return launch_chi_m2(pois, dich, gauss, P, K, n_steps, ws, bt, gb, sm, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_point(int model, bool pois, int dich, int gauss, int ppt, const PointConsts& P,
                         const LaunchConsts& K, const Workspace& ws, const PathOutPtrs& po,
                         int bt, int gb, int sm, cudaStream_t st)
{
#define SDE_M(M) \
    case M: return ppt == 2 ? launch_point_m##M##_p2(pois, dich, gauss, P, K, ws, po, bt, gb, sm, st) \
                            : launch_point_m##M##_p1(pois, dich, gauss, P, K, ws, po, bt, gb, sm, st);
    switch (model) {
    SDE_M(0) SDE_M(1) SDE_M(2)
    default: return cudaErrorInvalidValue;
    }
#undef SDE_M
}

cudaError_t launch_segment(int model, bool pois, int dich, int gauss, const PointConsts& P,
                           const LaunchConsts& K, const StatePlanes& M, uint32_t na, uint32_t nb,
                           const Workspace& ws, const PathOutPtrs& po, int bt, int gb, int sm,
                           cudaStream_t st)
{
    switch (model) {
    case kModelInertial: return launch_segment_m0(pois, dich, gauss, P, K, M, na, nb, ws, po, bt, gb, sm, st);
    case kModelOverdampedWashboard:
        return launch_segment_m1(pois, dich, gauss, P, K, M, na, nb, ws, po, bt, gb, sm, st);
    case kModelPWL: return launch_segment_m2(pois, dich, gauss, P, K, M, na, nb, ws, po, bt, gb, sm, st);
    default: return cudaErrorInvalidValue;
    }
}

int point_blocks_per_sm(int model, bool pois, int dich, int gauss, int ppt, int bt)
{
#define SDE_M(M) \
    case M: return ppt == 2 ? blocks_per_sm_m##M##_p2(pois, dich, gauss, bt) \
                            : blocks_per_sm_m##M##_p1(pois, dich, gauss, bt);
    switch (model) {
    SDE_M(0) SDE_M(1) SDE_M(2)
    default: return 0;
    }
#undef SDE_M
}

// ---------------------------------------------------------------- batched scan

// Persistent scan over (point, 32-path tile) items of the inertial washboard
// (Sec. 5: many parameter values in one kernel call).  Items are ordered
// longest first on the host; each warp pulls the next one from the counter.
// Six resident blocks per SM (at most 80 registers): the per-point constants
// live in registers here, and without the bound the kernel takes 96 (five
// blocks); measured 0.5-1 % faster despite a few spilled bytes.
template <bool POIS, int DICH, int GAUSS>
__global__ void __launch_bounds__(128, 6) scan_kernel(const PointConsts* __restrict__ pts,
                                                   const uint2* __restrict__ items,
                                                   const __grid_constant__ LaunchConsts K,
                                                   uint32_t* __restrict__ counter,
                                                   int32_t* __restrict__ status,
                                                   double* __restrict__ partials)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t t0 = K.budget_ns ? globaltimer_ns() : 0ull;
    constexpr bool kKickWin = WindowedKicks<POIS, GAUSS>::value;
    uint32_t* win = nullptr;
    if constexpr (kKickWin) {
        extern __shared__ uint32_t sde_scan1_smem[];
        win = sde_scan1_smem + (threadIdx.x >> 5) * kKickWordsPerWarp + lane;
    }
    for (;;) {
        const uint32_t item = next_item(counter, status, K, lane, t0);
        if (item == 0xffffffffu) break;
        const uint2 it = items[item];
        const PointConsts P = pts[it.x];
        const uint32_t path = it.y + lane;
        const bool valid = path < P.n_paths;
        PathResult R;
        simulate_path<kModelInertial, POIS, DICH, GAUSS, kKickWin>(P, K, path, lane, R, win);
        store_partial(partials, item, lane, valid, R);
    }
}

template <bool POIS, int DICH, int GAUSS>
static cudaError_t launch_scan_t(const PointConsts* pts, const uint2* items, const LaunchConsts& K,
                                 const Workspace& ws, int bt, int gb, int sm, cudaStream_t st)
{
    auto kern = scan_kernel<POIS, DICH, GAUSS>;
    const size_t smem = WindowedKicks<POIS, GAUSS>::value
                            ? (size_t)(bt / 32) * kKickWordsPerWarp * sizeof(uint32_t) : 0u;
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

cudaError_t launch_scan(bool pois, int dich, int gauss, const PointConsts* pts, const uint2* items,
                        const LaunchConsts& K, const Workspace& ws, int bt, int gb, int sm,
                        cudaStream_t st)
{
#define SDE_SCAN(PO, DI, GA) \
    if (pois == PO && dich == DI && gauss == GA) \
        return launch_scan_t<PO, DI, GA>(pts, items, K, ws, bt, gb, sm, st);
    SDE_SCAN(true, 1, kGauss3Point) SDE_SCAN(true, 0, kGauss3Point) SDE_SCAN(true, 2, kGauss3Point)
    SDE_SCAN(false, 1, kGauss3Point) SDE_SCAN(false, 0, kGauss3Point) SDE_SCAN(false, 2, kGauss3Point)
    SDE_SCAN(true, 1, 0) SDE_SCAN(true, 0, 0) SDE_SCAN(true, 2, 0)
    SDE_SCAN(false, 1, 0) SDE_SCAN(false, 0, 0) SDE_SCAN(false, 2, 0)
#undef SDE_SCAN
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- FP64 fold

// One block per point: thread t Kahan-sums items t, t + 256, ... in order,
// then a fixed pairwise tree over the 256 thread sums.  The result depends
// only on the partials, never on scheduling.
__global__ void __launch_bounds__(256) fold_kernel(const double* __restrict__ partials,
                                                   const uint2* __restrict__ ranges,
                                                   double* __restrict__ out5)
{
    __shared__ double sh[5][256];
    const uint2 r = ranges[blockIdx.x];
    const uint32_t t = threadIdx.x;
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double c[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (uint32_t i = t; i < r.y; i += 256u) {
        const double* p = partials + 5ull * (r.x + i);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const double y = p[q] - c[q];
            const double z = s[q] + y;
            c[q] = (z - s[q]) - y;
            s[q] = z;
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) sh[q][t] = s[q] - c[q];
    __syncthreads();
    for (uint32_t w = 128u; w > 0u; w >>= 1) {
        if (t < w) {
#pragma unroll
            for (int q = 0; q < 5; ++q) sh[q][t] += sh[q][t + w];
        }
        __syncthreads();
    }
    if (t < 5u) out5[5ull * blockIdx.x + t] = sh[t][0];
}

cudaError_t launch_fold(const double* partials, const uint2* ranges, uint32_t npts, double* out5,
                        cudaStream_t st)
{
    if (npts == 0) return cudaSuccess;
    fold_kernel<<<npts, 256, 0, st>>>(partials, ranges, out5);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reductions

__global__ void __launch_bounds__(256) reduce_items_kernel(const double* __restrict__ vals,
                                                           uint64_t n, double* __restrict__ partials)
{
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t i = gw * 32ull + lane;
    const bool valid = i < n;
    const double v = valid ? vals[i] : 0.0;
    const double a = warp_sum(valid ? 1.0 : 0.0);
    const double b = warp_sum(v);
    const double c = warp_sum(__dmul_rn(v, v));
    if (lane == 0u && gw * 32ull < n) {
        double* o = partials + 5ull * gw;
        o[0] = a; o[1] = b; o[2] = c; o[3] = 0.0; o[4] = 0.0;
    }
}

cudaError_t launch_reduce_items(const double* vals, uint64_t n, double* partials, cudaStream_t st)
{
    const uint64_t items = (n + 31ull) / 32ull;
    const uint64_t blocks = (items * 32ull + 255ull) / 256ull;
    if (blocks == 0) return cudaSuccess;
    reduce_items_kernel<<<(unsigned)blocks, 256, 0, st>>>(vals, n, partials);
    return cudaGetLastError();
}

__global__ void philox_kernel(const uint4* __restrict__ ctr, uint64_t n,
                              const __grid_constant__ LaunchConsts K, uint4* __restrict__ out)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox10(ctr[i], K);
}

cudaError_t launch_philox(const uint4* ctr, uint64_t n, const LaunchConsts& K, uint4* out,
                          cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, n, K, out);
    return cudaGetLastError();
}

}  // namespace sde
