// noalloc.cu -- sde_run_noalloc: a Monte Carlo run that allocates nothing.
//
// For callers that must not allocate device memory: code running under a
// memory pool or arena that owns every allocation, real-time loops that may
// not call cudaMalloc/cudaFree (both can synchronise the device), and hosts
// that forbid allocation after start-up.  The engine's scratch (work counter,
// status word, fold range and the per-item FP64 partial sums) lives in one
// file-scope device array of fixed size instead of the context's workspace.
#include <cstring>
#include <mutex>

#include "sde.h"
#include "capi_internal.h"
#include "launch.h"

using namespace sde;

namespace {

constexpr uint32_t kNoAllocMaxItems = SDE_NOALLOC_MAX_PATHS / 32u;
constexpr size_t kPartialsOffset = 256;          // counter, status, fold range first
constexpr size_t kScratchBytes = kPartialsOffset + 5u * sizeof(double) * kNoAllocMaxItems;

// The scratch array.  Every GPU that loads this library holds it until the
// process exits.  In host code its name is only a host-side stand-in; the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on each device does this set-up).
cudaError_t scratch_address(int device, void** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[device] = p;
    }
    *out = g_scratch_dev[device];
    return cudaSuccess;
}

// Clears what must start at zero (the array keeps the previous call's
// contents) and writes the fold range of the single point.
__global__ void noalloc_begin(uint32_t* counter, int32_t* status, uint2* range, uint32_t n_items)
{
    *counter = 0u;
    *status = kStatusOk;
    *range = make_uint2(0u, n_items);
}

__global__ void noalloc_end(const int32_t* status, int32_t* status_out)
{
    *status_out = *status;
}

}  // namespace

extern "C" int sde_run_noalloc(sde_model model, const sde_params* p, uint64_t seed, uint64_t paths,
                               double dt, uint64_t n_transient, uint64_t n_avg, void* cuda_stream,
                               double* out5, int32_t* status_out)
{
    int rc = validate_params(nullptr, model, p);
    if (rc) return rc;
    if ((rc = validate_run(nullptr, paths, dt, n_transient, n_avg))) return rc;
    if (paths > SDE_NOALLOC_MAX_PATHS)
        return fail(nullptr, SDE_EINVAL, "sde_run_noalloc: paths exceeds SDE_NOALLOC_MAX_PATHS (2^21)");
    if (!out5) return fail(nullptr, SDE_EINVAL, "sde_run_noalloc: out5 is NULL");
    int device = 0, sm_count = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess && (device < 0 || device >= kMaxDevices)) e = cudaErrorInvalidDevice;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device);
    void* base = nullptr;
    if (e == cudaSuccess) e = scratch_address(device, &base);
    if (e != cudaSuccess)
        return fail(nullptr, SDE_ECUDA, std::string("sde_run_noalloc set-up: ") + cudaGetErrorString(e));
    PointConsts P;
    if ((rc = make_point(nullptr, model, *p, dt, paths, n_transient, n_avg, P))) return rc;
    const uint32_t items = (uint32_t)((paths + 31ull) / 32ull);
    const LaunchConsts K = make_launch(seed, items, 0);
    char* b = (char*)base;
    Workspace ws{(uint32_t*)b, (int32_t*)(b + 4), (double*)(b + kPartialsOffset)};
    uint2* range = (uint2*)(b + 8);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const uint32_t f = p->noise_flags;
    PathOutPtrs po{nullptr, nullptr, nullptr, nullptr, nullptr};
    noalloc_begin<<<1, 1, 0, st>>>(ws.counter, ws.status, range, items);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_point((int)model, (f & SDE_NOISE_POISSON) != 0, dich_kind(f),
                         gauss_kind(*p), 1, P, K, ws, po, 128, 0, sm_count, st);
    if (e == cudaSuccess) e = launch_fold(ws.partials, range, 1, out5, st);
    if (e == cudaSuccess && status_out) {
        noalloc_end<<<1, 1, 0, st>>>(ws.status, status_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fail(nullptr, SDE_ECUDA, std::string("sde_run_noalloc launch: ") + cudaGetErrorString(e));
    return SDE_OK;
}
