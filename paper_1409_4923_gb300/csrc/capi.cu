// capi.cu -- host runtime of the engine behind the C ABI of include/sde.h.
//
// The context validates parameters, turns them into FP32/FP64 kernel
// constants once (in FP64 on the host), owns a grow-only device workspace and
// a pinned result buffer, and enqueues: counter reset -> persistent path
// kernel -> fixed-order FP64 fold -> 40-byte device-to-host copy.  It also
// runs batched scans (graph-replayed, resumable after a deadline), segmented
// runs with host checkpoints, and the local-error diagnostic.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "sde.h"
#include "capi_internal.h"
#include "launch.h"

using namespace sde;

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr uint32_t kMaxSteps = 0x7FFFFF00u;   // n_transient + n_avg: event steps stay below 2^32

struct ScanGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// What sde_scan_resume needs of a scan that ran out of time.
struct PendingScan {
    bool pending = false;
    uint64_t gen = 0;
    uint32_t npts = 0;
    uint32_t flags = 0;
    uint32_t total_items = 0;
    bool scan_kernel = false;
    bool x2 = false;              // two paths per lane (64-path items)
    int ppt = 1;                  // paths per lane of the per-point launches
    std::vector<uint32_t> order;  // their launch order
    size_t off_counters = 0, off_out5 = 0, off_ranges = 0, off_partials = 0, off_pts = 0,
           off_items = 0;
    std::vector<uint64_t> n_avg;
    std::vector<uint2> ranges;
    std::vector<PointConsts> P;
    std::vector<int> gauss;
};

struct SegmentedRun {
    bool active = false;
    sde_params p{};
    uint64_t seed = 0;
    uint64_t paths = 0, n_tr = 0, n_avg = 0, n_done = 0;
    double dt = 0.0;
    uint32_t items = 0, stride = 0;
};

// Checkpoint header (host byte order; followed by the saved states).
struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t model;
    uint64_t seed;
    sde_params p;
    double dt;
    uint64_t paths, n_tr, n_avg, n_done;
    uint32_t stride, bytes_per_path;
    uint64_t state_bytes;
    uint64_t checksum;
};
static_assert(sizeof(CkptHeader) == 224, "checkpoint header layout");
constexpr char kCkptMagic[8] = {'S', 'D', 'E', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 1;

// FNV-1a, 64 bit.
uint64_t fnv1a64(const unsigned char* p, size_t n)
{
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

}  // namespace

struct sde_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    sde_model model = SDE_INERTIAL_WASHBOARD;
    sde_params p{};
    uint64_t seed = 0;
    std::string err;
    // device workspace
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // pinned host results
    double* host = nullptr;
    size_t host_bytes = 0;
    cudaEvent_t done = nullptr;
    bool has_run = false;
    uint64_t last_paths = 0;
    uint64_t last_n_avg = 0;
    // tuning
    int block_threads = 128;
    int grid_blocks = 0;          // 0 = persistent grid from occupancy
    int paths_per_thread = 1;     // paths integrated by one lane, interleaved
    uint64_t steps_per_launch = 0;   // 0 = a whole run per launch
    void* run_state = nullptr;    // saved states of runs cut into launches
    size_t run_state_bytes = 0;
    // scan graphs keyed by (npts, n_items, flags, budget)
    // (and the caller's device output array of sde_scan_device, 0 for sde_scan)
    std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint64_t, uint64_t>, ScanGraph> graphs;
    // bumped by every call that writes the workspace; a timed-out scan can be
    // resumed only while its workspace is untouched
    uint64_t ws_gen = 0;
    PendingScan scan;
    // side streams and events of scans run as one point-kernel launch per point
    std::vector<cudaStream_t> fan;
    std::vector<cudaEvent_t> fan_ev;
    int scan_mode = 0;            // 0 automatic, 1 persistent scan kernel, 2 one launch per point
    // segmented run and its saved path states (device)
    SegmentedRun seg;
    void* state = nullptr;
    size_t state_bytes = 0;
};

// Message of the last failed call made without a context (sde_create,
// sde_run_noalloc): one per host thread, so that threads do not race on it.
static thread_local std::string g_create_error;

int fail(sde_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg; else g_create_error = msg;
    return code;
}

static int cuda_fail(sde_ctx* c, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? SDE_ENOMEM : SDE_ECUDA, m);
}

#define SDE_CUDA(c, call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); } while (0)

static bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

int validate_params(sde_ctx* c, sde_model model, const sde_params* p)
{
    if (!p) return fail(c, SDE_EINVAL, "params is NULL");
    if ((int)model < 0 || (int)model > 2) return fail(c, SDE_EINVAL, "unknown model");
    const double all[] = {p->gamma, p->a, p->omega, p->F, p->Q, p->lambda, p->zeta, p->Fa, p->Fb,
                          p->mua, p->mub, p->V0, p->x0_lo, p->x0_hi, p->v0_lo, p->v0_hi};
    for (double x : all)
        if (!std::isfinite(x)) return fail(c, SDE_EINVAL, "non-finite parameter");
    if (!finite_nonneg(p->Q)) return fail(c, SDE_EINVAL, "Q must be >= 0");
    if (model == SDE_INERTIAL_WASHBOARD && !(p->gamma > 0.0))
        return fail(c, SDE_EINVAL, "gamma must be > 0 for the inertial model");
    if (p->noise_flags & ~63u) return fail(c, SDE_EINVAL, "unknown noise flag");
    if ((p->noise_flags & SDE_DICHOT_IN_DRIFT) && !(p->noise_flags & SDE_NOISE_DICHOT))
        return fail(c, SDE_EINVAL, "SDE_DICHOT_IN_DRIFT needs SDE_NOISE_DICHOT");
    if ((p->noise_flags & SDE_NOISE_POISSON) && !(p->lambda > 0.0 && p->zeta > 0.0))
        return fail(c, SDE_EINVAL, "Poisson noise needs lambda > 0 and zeta > 0");
    if ((p->noise_flags & SDE_NOISE_DICHOT) &&
        !(p->mua > 0.0 && p->mub > 0.0 && p->Fa >= 0.0 && p->Fb >= 0.0))
        return fail(c, SDE_EINVAL, "dichotomous noise needs mua, mub > 0 and Fa, Fb >= 0");
    if (p->point >= (1u << 30)) return fail(c, SDE_EINVAL, "point id must be < 2^30");
    return SDE_OK;
}

int validate_run(sde_ctx* c, uint64_t paths, double dt, uint64_t n_tr, uint64_t n_avg)
{
    if (paths < 1 || paths > 0xFFFFFFC0ull) return fail(c, SDE_EINVAL, "paths must be in [1, 2^32 - 64]");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, SDE_EINVAL, "dt must be finite and > 0");
    if (n_avg < 1) return fail(c, SDE_EINVAL, "n_avg must be >= 1");
    if (n_tr > kMaxSteps || n_avg > kMaxSteps || n_tr + n_avg > kMaxSteps)
        return fail(c, SDE_EINVAL, "n_transient + n_avg must be < 2^31 - 256");
    return SDE_OK;
}

// Gaussian kernel variant: none (flag off or zero intensity), three-point, Gaussian.
// Dichotomous kernel variant: none, corrector increment (Algorithm 1), or drift term.
int dich_kind(uint32_t flags)
{
    if (!(flags & SDE_NOISE_DICHOT)) return 0;
    return (flags & SDE_DICHOT_IN_DRIFT) ? 2 : 1;
}

int gauss_kind(const sde_params& p)
{
    if (!(p.noise_flags & SDE_NOISE_GAUSS) || !(p.Q > 0.0)) return 0;
    return (p.noise_flags & SDE_GAUSS_NORMAL) ? kGaussNormal : kGauss3Point;
}

// Kernel constants of one point, from the FP64 parameters.  Coordinates:
// washboards integrate c = 2 pi x (so the SFU cosine takes c directly), the
// piecewise-linear model integrates x; noise is scaled into those units.
int make_point(sde_ctx* c, sde_model model, const sde_params& p, double dt, uint64_t paths,
                      uint64_t n_tr, uint64_t n_avg, PointConsts& P)
{
    std::memset(&P, 0, sizeof(P));
    const bool inertial = model == SDE_INERTIAL_WASHBOARD;
    const bool pwl = model == SDE_OVERDAMPED_PWL;
    const double cs = pwl ? 1.0 : kTwoPi;             // coordinate per unit x
    const double ns = inertial ? 1.0 : cs;            // noise acts on v (inertial) or the coordinate
    const uint32_t f = p.noise_flags;

    P.gdt = (float)(p.gamma * dt);
    if (inertial) P.fdt = (float)(p.V0 * kTwoPi * dt);
    else if (pwl) P.fdt = (float)(p.V0 * dt);
    else P.fdt = (float)(p.V0 * kTwoPi * cs * dt);
    P.wdt = (float)(cs * dt);
    P.whdt = (float)(0.5 * cs * dt);
    const double dscale = inertial ? dt : cs * dt;
    P.a_dt = (float)(p.a * dscale);
    P.F_dt = (float)(p.F * dscale);
    double frac = p.omega * dt / kTwoPi;
    frac -= std::floor(frac);
    double fx = std::ldexp(frac, 64);
    P.phase_step = fx >= 18446744073709551615.0 ? 0ull : (uint64_t)fx;

    const double G = inertial ? std::sqrt(2.0 * p.gamma * p.Q) : std::sqrt(2.0 * p.Q);
    P.xi_c = (float)(ns * G * ((f & SDE_GAUSS_NORMAL) ? std::sqrt(dt) : std::sqrt(3.0 * dt)));
    if (f & SDE_NOISE_POISSON) {
        const double aP = (f & SDE_POIS_COMPENSATED) ? p.zeta * (-std::expm1(-p.lambda * dt)) / dt
                                                     : p.lambda * p.zeta;
        if (p.lambda * dt < 2e-8) return fail(c, SDE_EINVAL, "lambda dt must be >= 2e-8");
        P.aP_dt = (float)(ns * aP * dt);
        P.zeta_l2 = (float)(ns * p.zeta * M_LN2);
        P.pois_cl2 = (float)(M_LN2 / (p.lambda * dt));
        P.inv_lambda = 1.0 / p.lambda;
    }
    if (f & SDE_NOISE_DICHOT) {
        if (p.mua * dt < 2e-8 || p.mub * dt < 2e-8) return fail(c, SDE_EINVAL, "mu dt must be >= 2e-8");
        P.Fb_dt = (float)(ns * p.Fb * dt);
        P.mFa_dt = (float)(-ns * p.Fa * dt);
        P.mua_cl2 = (float)(M_LN2 / (p.mua * dt));
        P.mub_cl2 = (float)(M_LN2 / (p.mub * dt));
        P.inv_mua = 1.0 / p.mua;
        P.inv_mub = 1.0 / p.mub;
        // d0 = F_b iff (w >> 8) 2^-24 < mua / (mua + mub)  <=>  (w >> 8) < ceil(thr 2^24)
        const double thr = p.mua / (p.mua + p.mub);
        P.d0_thresh = (uint32_t)std::ceil(std::ldexp(thr, 24));
    }
    P.dt64 = dt;
    P.x0_lo = (float)p.x0_lo;
    P.x0_span = (float)(p.x0_hi - p.x0_lo);
    P.v0_lo = (float)p.v0_lo;
    P.v0_span = (float)(p.v0_hi - p.v0_lo);
    P.c1_init = (kTagInit << 30) | p.point;
    P.c1_gauss = (kTagGauss << 30) | p.point;
    P.c1_pois = (kTagPois << 30) | p.point;
    P.c1_dich = (kTagDich << 30) | p.point;
    P.n_tr = (uint32_t)n_tr;
    P.n_avg = (uint32_t)n_avg;
    P.n_paths = (uint32_t)paths;
    P.inv_window = 1.0 / ((double)n_avg * dt);
    // the fold subtracts FP32 multiples of the period constant; the unfolded
    // coordinate therefore advances by that constant per folded period
    P.period = pwl ? 2.0 : (double)6.2831853071795865f / kTwoPi;
    P.coord_to_x = pwl ? 1.0 : 1.0 / kTwoPi;
    return SDE_OK;
}

LaunchConsts make_launch(uint64_t seed, uint32_t n_items, uint64_t budget_ns)
{
    LaunchConsts K;
    std::memset(&K, 0, sizeof(K));
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.rk0[r] = k0;
        K.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    K.n_items = n_items;
    K.budget_ns = budget_ns;
    return K;
}

// Cached scan graphs bake workspace and pinned-buffer addresses and the
// launch shape; dropped (after the stream drains) when any of them changes.
static void drop_graphs(sde_ctx* c)
{
    if (c->graphs.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto& kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    c->graphs.clear();
}

static int ensure_ws(sde_ctx* c, size_t bytes)
{
    if (bytes <= c->ws_bytes) return SDE_OK;
    drop_graphs(c);
    if (c->ws) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    size_t want = std::max(bytes, c->ws_bytes * 2);
    SDE_CUDA(c, cudaMalloc(&c->ws, want));
    c->ws_bytes = want;
    return SDE_OK;
}

static int ensure_host(sde_ctx* c, size_t bytes)
{
    if (bytes <= c->host_bytes) return SDE_OK;
    drop_graphs(c);
    if (c->host) {
        cudaStreamSynchronize(c->stream);
        cudaFreeHost(c->host);
        c->host = nullptr;
        c->host_bytes = 0;
    }
    SDE_CUDA(c, cudaMallocHost((void**)&c->host, bytes));
    c->host_bytes = bytes;
    return SDE_OK;
}

static size_t align256(size_t x) { return (x + 255u) & ~(size_t)255u; }

// Workspace layout: [counter u32, status i32 | ranges uint2[npts] | out5 f64[5 npts] |
//                    partials f64[5 items] | extra]
struct Layout {
    size_t off_ranges, off_out5, off_partials, off_extra, total;
};

static Layout layout(uint32_t npts, uint64_t items, size_t extra)
{
    Layout L;
    L.off_ranges = 256;
    L.off_out5 = L.off_ranges + align256(sizeof(uint2) * npts);
    L.off_partials = L.off_out5 + align256(sizeof(double) * 5 * npts);
    L.off_extra = L.off_partials + align256(sizeof(double) * 5 * items);
    L.total = L.off_extra + align256(extra);
    return L;
}

static void fill_stats(const double* s5, int32_t status, uint64_t n_avg, sde_stats_t* o)
{
    std::memset(o, 0, sizeof(*o));
    for (int i = 0; i < 5; ++i) o->sums[i] = s5[i];
    const double n = s5[0];
    o->n = (uint64_t)n;
    if (n > 0) {
        o->mean_v = s5[1] / n;
        o->var_v = n > 1 ? std::max(0.0, (s5[2] - n * o->mean_v * o->mean_v) / (n - 1.0)) : 0.0;
        o->stderr_v = std::sqrt(o->var_v / n);
        const double cnt = n * (double)n_avg;
        o->tmean_v = s5[3] / cnt;
        o->tvar_v = s5[4] / cnt - o->tmean_v * o->tmean_v;
    }
    o->status = status;
}

extern "C" {

const char* sde_version(void) { return "sde-gb300 1.0 (sm_103a)"; }

const char* sde_last_error(const sde_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int sde_create(sde_ctx** out, sde_model model, const sde_params* p, uint64_t seed, void* cuda_stream)
{
    if (!out) return fail(nullptr, SDE_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_params(nullptr, model, p);
    if (rc) return rc;
    sde_ctx* c = new (std::nothrow) sde_ctx();
    if (!c) return fail(nullptr, SDE_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess && cuda_stream == nullptr) {
        e = cudaStreamCreate(&c->stream);
        c->own_stream = e == cudaSuccess;
    } else {
        c->stream = (cudaStream_t)cuda_stream;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "sde_create");
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return e == cudaErrorMemoryAllocation ? SDE_ENOMEM : SDE_ECUDA;
    }
    c->model = model;
    c->p = *p;
    c->seed = seed;
    *out = c;
    return SDE_OK;
}

int sde_set_params(sde_ctx* c, const sde_params* p)
{
    if (!c) return SDE_EINVAL;
    int rc = validate_params(c, c->model, p);
    if (rc) return rc;
    c->p = *p;
    return SDE_OK;
}

int sde_set_tuning(sde_ctx* c, int block_threads, int grid_blocks)
{
    if (!c) return SDE_EINVAL;
    if (block_threads < 32 || block_threads > 128 || block_threads % 32)
        return fail(c, SDE_EINVAL, "block_threads must be 32, 64, 96 or 128");
    if (grid_blocks < 0) return fail(c, SDE_EINVAL, "grid_blocks must be >= 0");
    if (block_threads != c->block_threads || grid_blocks != c->grid_blocks) drop_graphs(c);
    c->block_threads = block_threads;
    c->grid_blocks = grid_blocks;
    return SDE_OK;
}

int sde_set_paths_per_thread(sde_ctx* c, int paths_per_thread)
{
    if (!c) return SDE_EINVAL;
    if (paths_per_thread != 1 && paths_per_thread != 2)
        return fail(c, SDE_EINVAL, "paths_per_thread must be 1 or 2");
    if (paths_per_thread != c->paths_per_thread) drop_graphs(c);
    c->paths_per_thread = paths_per_thread;
    return SDE_OK;
}

int sde_set_scan_mode(sde_ctx* c, int mode)
{
    if (!c) return SDE_EINVAL;
    if (mode < 0 || mode > 2) return fail(c, SDE_EINVAL, "scan mode must be 0, 1 or 2");
    c->scan_mode = mode;
    return SDE_OK;
}

int sde_set_steps_per_launch(sde_ctx* c, uint64_t steps)
{
    if (!c) return SDE_EINVAL;
    if (steps % 32u != 0u || steps > kMaxSteps)
        return fail(c, SDE_EINVAL, "steps_per_launch must be a multiple of 32 (0 = whole run)");
    c->steps_per_launch = steps;
    return SDE_OK;
}

int sde_occupancy(sde_ctx* c, int block_threads, int* blocks_per_sm, int* sm_count)
{
    if (!c || !blocks_per_sm || !sm_count) return SDE_EINVAL;
    const uint32_t f = c->p.noise_flags;
    *blocks_per_sm = point_blocks_per_sm((int)c->model, (f & SDE_NOISE_POISSON) != 0,
                                         dich_kind(f), gauss_kind(c->p),
                                         c->paths_per_thread, block_threads);
    *sm_count = c->sm_count;
    return SDE_OK;
}

static int run_impl(sde_ctx* c, uint64_t first_path, uint64_t paths, double dt, uint64_t n_tr,
                    uint64_t n_avg, const sde_path_out* out)
{
    if (!c) return SDE_EINVAL;
    int rc = validate_run(c, paths, dt, n_tr, n_avg);
    if (rc) return rc;
    if (first_path > 0xFFFFFFFFull || first_path + ((paths + 31ull) & ~31ull) > 0x100000000ull)
        return fail(c, SDE_EINVAL, "first_path + paths must stay within the 32-bit path counter");
    const uint64_t items = (paths + 31ull) / 32ull;
    PointConsts P;
    rc = make_point(c, c->model, c->p, dt, paths, n_tr, n_avg, P);
    if (rc) return rc;
    P.path0 = (uint32_t)first_path;
    const Layout L = layout(1, items, 0);
    if ((rc = ensure_ws(c, L.total))) return rc;
    if ((rc = ensure_host(c, 64))) return rc;
    ++c->ws_gen;
    char* base = (char*)c->ws;
    Workspace ws{(uint32_t*)base, (int32_t*)(base + 4), (double*)(base + L.off_partials)};
    uint2* ranges = (uint2*)(base + L.off_ranges);
    double* out5 = (double*)(base + L.off_out5);
    const uint2 r0 = make_uint2(0u, (uint32_t)items);
    SDE_CUDA(c, cudaMemsetAsync(base, 0, 8, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(ranges, &r0, sizeof(r0), cudaMemcpyHostToDevice, c->stream));
    PathOutPtrs po{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (out) po = PathOutPtrs{out->X_f, out->v_f, out->vbar, out->jP, out->jD};
    const LaunchConsts K = make_launch(c->seed, (uint32_t)items, 0);
    const uint32_t f = c->p.noise_flags;
    const uint64_t total = n_tr + n_avg;
    if (c->steps_per_launch == 0 || c->steps_per_launch >= total) {
        SDE_CUDA(c, launch_point((int)c->model, (f & SDE_NOISE_POISSON) != 0, dich_kind(f),
                                 gauss_kind(c->p), c->paths_per_thread, P, K, ws, po, c->block_threads,
                                 c->grid_blocks, c->sm_count, c->stream));
    } else {
        // Algorithm 5 with `samples` = steps_per_launch: the path states stay
        // in device memory between launches; cut points are multiples of 32
        // steps, so the results are those of one launch bit for bit
        const size_t need = (size_t)kStateBytesPerPath * items * 32ull;
        if (need > c->run_state_bytes) {
            if (c->run_state) {
                cudaStreamSynchronize(c->stream);
                cudaFree(c->run_state);
                c->run_state = nullptr;
                c->run_state_bytes = 0;
            }
            SDE_CUDA(c, cudaMalloc(&c->run_state, need));
            c->run_state_bytes = need;
        }
        const StatePlanes M{(unsigned char*)c->run_state, (uint32_t)(items * 32ull)};
        for (uint64_t na = 0; na < total; na += c->steps_per_launch) {
            const uint64_t nb = std::min(total, na + c->steps_per_launch);
            if (na > 0) SDE_CUDA(c, cudaMemsetAsync(base, 0, 4, c->stream));
            SDE_CUDA(c, launch_segment((int)c->model, (f & SDE_NOISE_POISSON) != 0,
                                       dich_kind(f), gauss_kind(c->p), P, K, M,
                                       (uint32_t)na, (uint32_t)nb, ws, po, c->block_threads,
                                       c->grid_blocks, c->sm_count, c->stream));
        }
    }
    SDE_CUDA(c, launch_fold(ws.partials, ranges, 1, out5, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(c->host, out5, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(c->host + 5, ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    SDE_CUDA(c, cudaEventRecord(c->done, c->stream));
    c->has_run = true;
    c->last_paths = paths;
    c->last_n_avg = n_avg;
    return SDE_OK;
}

int sde_run(sde_ctx* c, uint64_t paths, double dt, uint64_t n_tr, uint64_t n_avg)
{
    return run_impl(c, 0, paths, dt, n_tr, n_avg, nullptr);
}

int sde_run_paths(sde_ctx* c, uint64_t paths, double dt, uint64_t n_tr, uint64_t n_avg,
                  const sde_path_out* out)
{
    return run_impl(c, 0, paths, dt, n_tr, n_avg, out);
}

int sde_run_range(sde_ctx* c, uint64_t first_path, uint64_t paths, double dt, uint64_t n_tr,
                  uint64_t n_avg, const sde_path_out* out)
{
    return run_impl(c, first_path, paths, dt, n_tr, n_avg, out);
}

int sde_stats(sde_ctx* c, sde_stats_t* out)
{
    if (!c || !out) return SDE_EINVAL;
    if (!c->has_run) return fail(c, SDE_ESTATE, "sde_stats before sde_run");
    SDE_CUDA(c, cudaEventSynchronize(c->done));
    int32_t status;
    std::memcpy(&status, c->host + 5, sizeof(status));
    fill_stats(c->host, status, c->last_n_avg, out);
    return status == kStatusOk ? SDE_OK : fail(c, SDE_ETIMEDOUT, "device deadline expired");
}

// One point-kernel launch per point of a scan, each with its own work
// counter (so that a timed-out scan can resume), spread over side streams
// forked from the context's stream and joined back to it: the launches run
// side by side, each with its point's constants as kernel arguments.  128
// streams: points of 2048 paths are eight 128-thread blocks each, and 64
// launches side by side left a third of the block slots empty (measured on
// 2048 such points: 2.12 s against 2.24 s with 64 streams).
constexpr int kFanStreams = 128;
constexpr uint64_t kPointScanMinPaths = 2048;

static int launch_points_fanout(sde_ctx* c, const std::vector<uint32_t>& order,
                                const std::vector<PointConsts>& P, const std::vector<uint2>& ranges,
                                const std::vector<int>& gauss, uint32_t flags, int ppt,
                                uint32_t* d_counters, const Workspace& ws, uint64_t budget)
{
    if (c->fan.empty()) {
        for (int k = 0; k < kFanStreams; ++k) {
            cudaStream_t st;
            SDE_CUDA(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            c->fan.push_back(st);
        }
        for (int k = 0; k <= kFanStreams; ++k) {
            cudaEvent_t ev;
            SDE_CUDA(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            c->fan_ev.push_back(ev);
        }
    }
    const int nfan = (int)std::min<size_t>(kFanStreams, order.size());
    SDE_CUDA(c, cudaEventRecord(c->fan_ev[kFanStreams], c->stream));
    for (int k = 0; k < nfan; ++k) SDE_CUDA(c, cudaStreamWaitEvent(c->fan[k], c->fan_ev[kFanStreams], 0));
    for (size_t k = 0; k < order.size(); ++k) {
        const uint32_t i = order[k];
        const LaunchConsts K = make_launch(c->seed, ranges[i].y, budget);
        Workspace wsi{d_counters + i, ws.status, ws.partials + 5ull * ranges[i].x};
        PathOutPtrs po{nullptr, nullptr, nullptr, nullptr, nullptr};
        SDE_CUDA(c, launch_point((int)c->model, (flags & SDE_NOISE_POISSON) != 0, dich_kind(flags), gauss[i],
                                 ppt, P[i], K, wsi, po, c->block_threads, c->grid_blocks, c->sm_count,
                                 c->fan[k % nfan]));
    }
    for (int k = 0; k < nfan; ++k) {
        SDE_CUDA(c, cudaEventRecord(c->fan_ev[k], c->fan[k]));
        SDE_CUDA(c, cudaStreamWaitEvent(c->stream, c->fan_ev[k], 0));
    }
    return SDE_OK;
}

// The batched scan.  Host mode (dev_out5 == NULL): statistics to the host
// array `out`, synchronising.  Device mode: each point's five FP64 sums to
// the caller's device array dev_out5, enqueued only (no deadline).
static int scan_impl(sde_ctx* c, const sde_scan_point* pts, uint32_t npts, sde_stats_t* out,
                     double deadline_ms, double* dev_out5)
{
    if (!c || (!pts && npts) || (!out && !dev_out5 && npts)) return SDE_EINVAL;
    if (npts == 0) return SDE_OK;
    if (!(deadline_ms >= 0.0) || !std::isfinite(deadline_ms)) return fail(c, SDE_EINVAL, "deadline_ms must be >= 0");
    const uint32_t flags = pts[0].p.noise_flags;
    std::vector<PointConsts> P(npts);
    std::vector<uint64_t> steps(npts);
    for (uint32_t i = 0; i < npts; ++i) {
        int rc = validate_params(c, c->model, &pts[i].p);
        if (rc) return rc;
        if (pts[i].p.noise_flags != flags) return fail(c, SDE_EINVAL, "all scan points need the same noise flags");
        if ((rc = validate_run(c, pts[i].paths, pts[i].dt, pts[i].n_transient, pts[i].n_avg))) return rc;
        steps[i] = pts[i].n_transient + pts[i].n_avg;
    }
    const uint64_t budget = (uint64_t)(deadline_ms * 1e6);
    // longest-processing-time-first order of points; items of a point stay contiguous
    std::vector<uint32_t> order(npts);
    for (uint32_t i = 0; i < npts; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return steps[a] > steps[b]; });
    // The inertial model runs either the persistent scan kernel or one point
    // kernel per point (side by side on side streams, with the point's
    // constants as kernel arguments, which the step loop reads from the
    // constant bank; in the scan kernel they compete for registers, and the
    // compiler reloads them from the point table inside the step loop).  With
    // 2048 paths per point on average the launches fill the GPU (up to 128 of
    // them side by side, 32 or more warps each) and run 8-12 % faster than the scan
    // kernel (measured on 256 and 512 dichotomous points of 8192 and 4096
    // paths, and on the 64 x 64 Poisson scan of 256 to 16384 paths); scans of
    // smaller points keep the persistent kernel.
    const bool inertial_scan = c->model == SDE_INERTIAL_WASHBOARD && !(flags & SDE_GAUSS_NORMAL);
    uint64_t sum_paths = 0;
    for (uint32_t i = 0; i < npts; ++i) sum_paths += pts[i].paths;
    // A deadline bounds each kernel's time from its own start, so a scan with a
    // deadline stays in the one persistent launch unless mode 2 is asked for.
    const bool use_scan_kernel =
        inertial_scan && (c->scan_mode == 1 ||
                          (c->scan_mode == 0 && (budget > 0 || sum_paths < kPointScanMinPaths * npts)));
    // Per-point launches of the inertial model take two paths per lane, with
    // Poisson noise too (measured on the 64 x 64 Poisson scan: 3.75 s against
    // 3.81 s with one path per lane).
    const int point_ppt = inertial_scan ? 2 : c->paths_per_thread;
    // Without Poisson noise the scan kernel takes two paths per lane: a work
    // item is 64 paths of one point and writes the partial records of its two
    // 32-path tiles, so each point's records start at an even index (a point
    // with an odd tile count leaves one record unused and unfolded).
    const bool x2 = use_scan_kernel && !(flags & SDE_NOISE_POISSON);
    const uint64_t item_paths = x2 ? 64ull : 32ull;
    std::vector<uint2> ranges(npts), items;
    uint64_t total_items = 0;
    for (uint32_t i = 0; i < npts; ++i) total_items += (pts[i].paths + item_paths - 1) / item_paths;
    if (total_items > 0x7FFFFF00ull) return fail(c, SDE_EINVAL, "too many work items");
    const uint64_t records = x2 ? 2 * total_items : total_items;
    items.reserve(total_items);
    for (uint32_t k = 0; k < npts; ++k) {
        const uint32_t i = order[k];
        const uint32_t first = (uint32_t)(x2 ? 2 * items.size() : items.size());
        const uint64_t ni = (pts[i].paths + item_paths - 1) / item_paths;
        for (uint64_t t = 0; t < ni; ++t) items.push_back(make_uint2(i, (uint32_t)(item_paths * t)));
        ranges[i] = make_uint2(first, (uint32_t)((pts[i].paths + 31ull) / 32ull));
        int rc = make_point(c, c->model, pts[i].p, pts[i].dt, pts[i].paths, pts[i].n_transient,
                            pts[i].n_avg, P[i]);
        if (rc) return rc;
    }
    const size_t off_items = align256(sizeof(PointConsts) * npts);
    const size_t off_counters = off_items + align256(sizeof(uint2) * total_items);
    const size_t extra = off_counters + align256(sizeof(uint32_t) * npts);
    const Layout L = layout(npts, records, extra);
    int rc;
    if ((rc = ensure_ws(c, L.total))) return rc;
    const size_t host_need = sizeof(double) * 5 * npts + 64;
    if ((rc = ensure_host(c, host_need))) return rc;
    c->scan.pending = false;
    const uint64_t gen = ++c->ws_gen;
    char* base = (char*)c->ws;
    Workspace ws{(uint32_t*)base, (int32_t*)(base + 4), (double*)(base + L.off_partials)};
    uint2* d_ranges = (uint2*)(base + L.off_ranges);
    double* d_out5 = (double*)(base + L.off_out5);
    PointConsts* d_pts = (PointConsts*)(base + L.off_extra);
    uint2* d_items = (uint2*)(base + L.off_extra + off_items);
    uint32_t* d_counters = (uint32_t*)(base + L.off_extra + off_counters);
    SDE_CUDA(c, cudaMemcpyAsync(d_pts, P.data(), sizeof(PointConsts) * npts, cudaMemcpyHostToDevice, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(d_items, items.data(), sizeof(uint2) * total_items, cudaMemcpyHostToDevice, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(d_ranges, ranges.data(), sizeof(uint2) * npts, cudaMemcpyHostToDevice, c->stream));
    double* h_out = c->host;
    int32_t* h_status = (int32_t*)(c->host + 5 * npts);
    if (use_scan_kernel) {
        const LaunchConsts K = make_launch(c->seed, (uint32_t)total_items, budget);
        auto key = std::make_tuple(npts, (uint32_t)total_items, flags, budget, (uint64_t)(uintptr_t)dev_out5);
        auto it = c->graphs.find(key);
        if (it == c->graphs.end() || c->stream == nullptr) {
            ScanGraph g;
            bool capture = c->stream != nullptr;
            if (capture) SDE_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaMemsetAsync(base, 0, 8, c->stream);
            if (e == cudaSuccess && x2)
                e = launch_scan_x2(dich_kind(flags), (flags & SDE_NOISE_GAUSS) ? kGauss3Point : 0, d_pts,
                                   d_items, K, ws, c->block_threads, c->grid_blocks, c->sm_count,
                                   c->stream);
            else if (e == cudaSuccess)
                e = launch_scan((flags & SDE_NOISE_POISSON) != 0, dich_kind(flags),
                                (flags & SDE_NOISE_GAUSS) ? kGauss3Point : 0, d_pts,
                                d_items, K, ws, c->block_threads, c->grid_blocks, c->sm_count, c->stream);
            if (e == cudaSuccess) e = launch_fold(ws.partials, d_ranges, npts, dev_out5 ? dev_out5 : d_out5, c->stream);
            if (e == cudaSuccess && !dev_out5)
                e = cudaMemcpyAsync(h_out, d_out5, sizeof(double) * 5 * npts, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess && !dev_out5)
                e = cudaMemcpyAsync(h_status, ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
            if (capture) {
                cudaError_t e2 = cudaStreamEndCapture(c->stream, &g.graph);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
                if (e != cudaSuccess) {
                    if (g.graph) cudaGraphDestroy(g.graph);
                    return cuda_fail(c, e, "scan graph capture");
                }
                c->graphs[key] = g;
                SDE_CUDA(c, cudaGraphLaunch(g.exec, c->stream));
            } else if (e != cudaSuccess) {
                return cuda_fail(c, e, "scan launch");
            }
        } else {
            SDE_CUDA(c, cudaGraphLaunch(it->second.exec, c->stream));
        }
    } else {
        // one point-kernel launch per point (each with its own work counter,
        // so that a timed-out scan can resume), longest first, same fold
        SDE_CUDA(c, cudaMemsetAsync(base + 4, 0, 4, c->stream));
        SDE_CUDA(c, cudaMemsetAsync(d_counters, 0, sizeof(uint32_t) * npts, c->stream));
        std::vector<int> gauss(npts);
        for (uint32_t i = 0; i < npts; ++i) gauss[i] = gauss_kind(pts[i].p);
        if ((rc = launch_points_fanout(c, order, P, ranges, gauss, flags, point_ppt, d_counters, ws, budget)))
            return rc;
        SDE_CUDA(c, launch_fold(ws.partials, d_ranges, npts, dev_out5 ? dev_out5 : d_out5, c->stream));
        if (!dev_out5) {
            SDE_CUDA(c, cudaMemcpyAsync(h_out, d_out5, sizeof(double) * 5 * npts, cudaMemcpyDeviceToHost, c->stream));
            SDE_CUDA(c, cudaMemcpyAsync(h_status, ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        }
    }
    if (dev_out5) return SDE_OK;          // device mode: enqueued only
    SDE_CUDA(c, cudaStreamSynchronize(c->stream));
    const int32_t status = *h_status;
    for (uint32_t i = 0; i < npts; ++i) fill_stats(h_out + 5ull * i, status, pts[i].n_avg, &out[i]);
    if (status == kStatusOk) return SDE_OK;
    PendingScan& S = c->scan;
    S.pending = true;
    S.gen = gen;
    S.npts = npts;
    S.flags = flags;
    S.total_items = (uint32_t)total_items;
    S.scan_kernel = use_scan_kernel;
    S.x2 = x2;
    S.ppt = point_ppt;
    S.order = order;
    S.off_counters = L.off_extra + off_counters;
    S.off_out5 = L.off_out5;
    S.off_ranges = L.off_ranges;
    S.off_partials = L.off_partials;
    S.off_pts = L.off_extra;
    S.off_items = L.off_extra + off_items;
    S.n_avg.resize(npts);
    S.gauss.resize(npts);
    for (uint32_t i = 0; i < npts; ++i) {
        S.n_avg[i] = pts[i].n_avg;
        S.gauss[i] = gauss_kind(pts[i].p);
    }
    S.ranges = ranges;
    S.P = P;
    return fail(c, SDE_ETIMEDOUT, "device deadline expired");
}

int sde_scan(sde_ctx* c, const sde_scan_point* pts, uint32_t npts, sde_stats_t* out, double deadline_ms)
{
    return scan_impl(c, pts, npts, out, deadline_ms, nullptr);
}

int sde_scan_device(sde_ctx* c, const sde_scan_point* pts, uint32_t npts, double* out5)
{
    if (c && npts && !out5) return fail(c, SDE_EINVAL, "out5 is NULL");
    return scan_impl(c, pts, npts, nullptr, 0.0, out5);
}

int sde_scan_resume(sde_ctx* c, sde_stats_t* out, double deadline_ms)
{
    if (!c || !out) return SDE_EINVAL;
    if (!(deadline_ms >= 0.0) || !std::isfinite(deadline_ms)) return fail(c, SDE_EINVAL, "deadline_ms must be >= 0");
    PendingScan& S = c->scan;
    if (!S.pending) return fail(c, SDE_ESTATE, "no timed-out scan to resume");
    if (S.gen != c->ws_gen) {
        S.pending = false;
        return fail(c, SDE_ESTATE, "the scan's workspace was used by another call");
    }
    const uint64_t budget = (uint64_t)(deadline_ms * 1e6);
    char* base = (char*)c->ws;
    Workspace ws{(uint32_t*)base, (int32_t*)(base + 4), (double*)(base + S.off_partials)};
    double* d_out5 = (double*)(base + S.off_out5);
    uint2* d_ranges = (uint2*)(base + S.off_ranges);
    double* h_out = c->host;
    int32_t* h_status = (int32_t*)(c->host + 5ull * S.npts);
    // the work counters keep the items already handed out (all of them finished)
    SDE_CUDA(c, cudaMemsetAsync(ws.status, 0, 4, c->stream));
    if (S.scan_kernel) {
        const LaunchConsts K = make_launch(c->seed, S.total_items, budget);
        if (S.x2)
            SDE_CUDA(c, launch_scan_x2(dich_kind(S.flags), (S.flags & SDE_NOISE_GAUSS) ? kGauss3Point : 0,
                                       (const PointConsts*)(base + S.off_pts),
                                       (const uint2*)(base + S.off_items), K, ws, c->block_threads,
                                       c->grid_blocks, c->sm_count, c->stream));
        else
            SDE_CUDA(c, launch_scan((S.flags & SDE_NOISE_POISSON) != 0, dich_kind(S.flags),
                                    (S.flags & SDE_NOISE_GAUSS) ? kGauss3Point : 0,
                                    (const PointConsts*)(base + S.off_pts), (const uint2*)(base + S.off_items),
                                    K, ws, c->block_threads, c->grid_blocks, c->sm_count, c->stream));
    } else {
        uint32_t* d_counters = (uint32_t*)(base + S.off_counters);
        int rc = launch_points_fanout(c, S.order, S.P, S.ranges, S.gauss, S.flags, S.ppt, d_counters, ws, budget);
        if (rc) return rc;
    }
    SDE_CUDA(c, launch_fold(ws.partials, d_ranges, S.npts, d_out5, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(h_out, d_out5, sizeof(double) * 5 * S.npts, cudaMemcpyDeviceToHost, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(h_status, ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    SDE_CUDA(c, cudaStreamSynchronize(c->stream));
    const int32_t status = *h_status;
    for (uint32_t i = 0; i < S.npts; ++i) fill_stats(h_out + 5ull * i, status, S.n_avg[i], &out[i]);
    if (status == kStatusOk) {
        S.pending = false;
        return SDE_OK;
    }
    return fail(c, SDE_ETIMEDOUT, "device deadline expired");
}

// ---------------------------------------------------------------- segmented runs

static int ensure_state(sde_ctx* c, size_t bytes)
{
    if (bytes <= c->state_bytes) return SDE_OK;
    if (c->state) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->state);
        c->state = nullptr;
        c->state_bytes = 0;
    }
    SDE_CUDA(c, cudaMalloc(&c->state, bytes));
    c->state_bytes = bytes;
    return SDE_OK;
}

static uint64_t seg_state_bytes(const SegmentedRun& r)
{
    return r.n_done ? (uint64_t)kStateBytesPerPath * r.stride : 0ull;
}

int sde_begin(sde_ctx* c, uint64_t paths, double dt, uint64_t n_tr, uint64_t n_avg)
{
    if (!c) return SDE_EINVAL;
    int rc = validate_run(c, paths, dt, n_tr, n_avg);
    if (rc) return rc;
    PointConsts P;
    if ((rc = make_point(c, c->model, c->p, dt, paths, n_tr, n_avg, P))) return rc;
    SegmentedRun r;
    r.p = c->p;
    r.seed = c->seed;
    r.paths = paths;
    r.dt = dt;
    r.n_tr = n_tr;
    r.n_avg = n_avg;
    r.n_done = 0;
    r.items = (uint32_t)((paths + 31ull) / 32ull);
    r.stride = r.items * 32u;
    if ((rc = ensure_state(c, (size_t)kStateBytesPerPath * r.stride))) return rc;
    r.active = true;
    c->seg = r;
    c->has_run = false;
    return SDE_OK;
}

int sde_advance(sde_ctx* c, uint64_t n_steps, const sde_path_out* out, uint64_t* n_done)
{
    if (!c) return SDE_EINVAL;
    SegmentedRun& r = c->seg;
    if (!r.active) return fail(c, SDE_ESTATE, "sde_advance without sde_begin or sde_restore");
    const uint64_t total = r.n_tr + r.n_avg;
    const uint64_t na = r.n_done;
    const uint64_t nb = (n_steps == 0 || n_steps >= total - na) ? total : na + n_steps;
    PointConsts P;
    int rc = make_point(c, c->model, r.p, r.dt, r.paths, r.n_tr, r.n_avg, P);
    if (rc) return rc;
    const Layout L = layout(1, r.items, 0);
    if ((rc = ensure_ws(c, L.total))) return rc;
    if ((rc = ensure_host(c, 64))) return rc;
    ++c->ws_gen;
    char* base = (char*)c->ws;
    Workspace ws{(uint32_t*)base, (int32_t*)(base + 4), (double*)(base + L.off_partials)};
    uint2* ranges = (uint2*)(base + L.off_ranges);
    double* out5 = (double*)(base + L.off_out5);
    const bool last = nb == total;
    SDE_CUDA(c, cudaMemsetAsync(base, 0, 8, c->stream));
    PathOutPtrs po{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (out && last) po = PathOutPtrs{out->X_f, out->v_f, out->vbar, out->jP, out->jD};
    const LaunchConsts K = make_launch(r.seed, r.items, 0);
    const StatePlanes M{(unsigned char*)c->state, r.stride};
    const uint32_t f = r.p.noise_flags;
    SDE_CUDA(c, launch_segment((int)c->model, (f & SDE_NOISE_POISSON) != 0, dich_kind(f),
                               gauss_kind(r.p), P, K, M, (uint32_t)na, (uint32_t)nb, ws, po,
                               c->block_threads, c->grid_blocks, c->sm_count, c->stream));
    if (last) {
        const uint2 r0 = make_uint2(0u, r.items);
        SDE_CUDA(c, cudaMemcpyAsync(ranges, &r0, sizeof(r0), cudaMemcpyHostToDevice, c->stream));
        SDE_CUDA(c, launch_fold(ws.partials, ranges, 1, out5, c->stream));
        SDE_CUDA(c, cudaMemcpyAsync(c->host, out5, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SDE_CUDA(c, cudaMemcpyAsync(c->host + 5, ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        SDE_CUDA(c, cudaEventRecord(c->done, c->stream));
        c->has_run = true;
        c->last_paths = r.paths;
        c->last_n_avg = r.n_avg;
    }
    r.n_done = nb;
    if (n_done) *n_done = nb;
    return SDE_OK;
}

int sde_checkpoint_size(sde_ctx* c, uint64_t* bytes)
{
    if (!c || !bytes) return SDE_EINVAL;
    if (!c->seg.active) return fail(c, SDE_ESTATE, "no segmented run");
    *bytes = sizeof(CkptHeader) + seg_state_bytes(c->seg);
    return SDE_OK;
}

int sde_checkpoint(sde_ctx* c, void* buf, uint64_t bytes)
{
    if (!c) return SDE_EINVAL;
    const SegmentedRun& r = c->seg;
    if (!r.active) return fail(c, SDE_ESTATE, "no segmented run");
    const uint64_t sb = seg_state_bytes(r);
    if (!buf || bytes < sizeof(CkptHeader) + sb) return fail(c, SDE_EINVAL, "checkpoint buffer too small");
    unsigned char* dst = (unsigned char*)buf + sizeof(CkptHeader);
    SDE_CUDA(c, cudaStreamSynchronize(c->stream));
    if (sb) {
        SDE_CUDA(c, cudaMemcpyAsync(dst, c->state, sb, cudaMemcpyDeviceToHost, c->stream));
        SDE_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = kCkptVersion;
    h.model = (uint32_t)c->model;
    h.seed = r.seed;
    h.p = r.p;
    h.dt = r.dt;
    h.paths = r.paths;
    h.n_tr = r.n_tr;
    h.n_avg = r.n_avg;
    h.n_done = r.n_done;
    h.stride = r.stride;
    h.bytes_per_path = kStateBytesPerPath;
    h.state_bytes = sb;
    h.checksum = fnv1a64(dst, sb);
    std::memcpy(buf, &h, sizeof(h));
    return SDE_OK;
}

int sde_restore(sde_ctx* c, const void* buf, uint64_t bytes)
{
    if (!c) return SDE_EINVAL;
    if (!buf || bytes < sizeof(CkptHeader)) return fail(c, SDE_EINVAL, "checkpoint too short");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0) return fail(c, SDE_EINVAL, "not a checkpoint");
    if (h.version != kCkptVersion) return fail(c, SDE_EINVAL, "unknown checkpoint version");
    if (h.model != (uint32_t)c->model) return fail(c, SDE_EINVAL, "checkpoint of another model");
    int rc = validate_params(c, c->model, &h.p);
    if (rc) return rc;
    if ((rc = validate_run(c, h.paths, h.dt, h.n_tr, h.n_avg))) return rc;
    SegmentedRun r;
    r.p = h.p;
    r.seed = h.seed;
    r.paths = h.paths;
    r.dt = h.dt;
    r.n_tr = h.n_tr;
    r.n_avg = h.n_avg;
    r.n_done = h.n_done;
    r.items = (uint32_t)((h.paths + 31ull) / 32ull);
    r.stride = r.items * 32u;
    if (h.n_done > h.n_tr + h.n_avg) return fail(c, SDE_EINVAL, "steps done exceed the run");
    if (h.stride != r.stride || h.bytes_per_path != kStateBytesPerPath)
        return fail(c, SDE_EINVAL, "checkpoint state layout mismatch");
    const uint64_t sb = seg_state_bytes(r);
    if (h.state_bytes != sb || bytes - sizeof(CkptHeader) < sb)
        return fail(c, SDE_EINVAL, "checkpoint truncated");
    const unsigned char* src = (const unsigned char*)buf + sizeof(CkptHeader);
    if (fnv1a64(src, sb) != h.checksum) return fail(c, SDE_EINVAL, "checkpoint checksum mismatch");
    PointConsts P;
    if ((rc = make_point(c, c->model, r.p, r.dt, r.paths, r.n_tr, r.n_avg, P))) return rc;
    if (sb) {
        // event counters: planes 0 (eP), 1 (JP), 4 (eD), 5 (JD), 6 (dst) of the u32 block
        const bool pois = (r.p.noise_flags & SDE_NOISE_POISSON) != 0;
        const bool dich = (r.p.noise_flags & SDE_NOISE_DICHOT) != 0;
        const unsigned char* u = src + 44ull * r.stride;
        auto word = [&](int plane, uint32_t i) {
            uint32_t w;
            std::memcpy(&w, u + 4ull * ((uint64_t)plane * r.stride + i), 4);
            return w;
        };
        for (uint32_t i = 0; i < r.stride; ++i) {
            if (pois && (word(0, i) < r.n_done || word(1, i) < 1u))
                return fail(c, SDE_EINVAL, "checkpoint: invalid Poisson event counter");
            if (dich && (word(4, i) < r.n_done || word(5, i) < 1u || word(6, i) > 1u))
                return fail(c, SDE_EINVAL, "checkpoint: invalid dichotomous event counter");
        }
    }
    if ((rc = ensure_state(c, (size_t)kStateBytesPerPath * r.stride))) return rc;
    if (sb) {
        SDE_CUDA(c, cudaMemcpyAsync(c->state, src, sb, cudaMemcpyHostToDevice, c->stream));
        SDE_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    r.active = true;
    c->seg = r;
    c->has_run = false;
    return SDE_OK;
}

int sde_local_error(sde_ctx* c, uint64_t paths, double dt, uint64_t n_steps, double* out4)
{
    if (!c || !out4) return SDE_EINVAL;
    int rc = validate_run(c, paths, dt, 0, n_steps);
    if (rc) return rc;
    PointConsts P;
    if ((rc = make_point(c, c->model, c->p, dt, paths, 0, n_steps, P))) return rc;
    const uint64_t items = (paths + 31ull) / 32ull;
    const Layout L = layout(1, items, 0);
    if ((rc = ensure_ws(c, L.total))) return rc;
    if ((rc = ensure_host(c, 5 * sizeof(double) * items + 64))) return rc;
    ++c->ws_gen;
    char* base = (char*)c->ws;
    Workspace ws{(uint32_t*)base, (int32_t*)(base + 4), (double*)(base + L.off_partials)};
    SDE_CUDA(c, cudaMemsetAsync(base, 0, 8, c->stream));
    const LaunchConsts K = make_launch(c->seed, (uint32_t)items, 0);
    const uint32_t f = c->p.noise_flags;
    SDE_CUDA(c, launch_chi((int)c->model, (f & SDE_NOISE_POISSON) != 0, dich_kind(f), gauss_kind(c->p), P, K,
                           (uint32_t)n_steps, ws, c->block_threads, c->grid_blocks, c->sm_count, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(c->host, ws.partials, 5 * sizeof(double) * items, cudaMemcpyDeviceToHost,
                                c->stream));
    SDE_CUDA(c, cudaStreamSynchronize(c->stream));
    double n = 0.0, sx = 0.0, sv = 0.0, mx = 0.0, mv = 0.0;
    for (uint64_t i = 0; i < items; ++i) {                  // fixed order
        const double* o = c->host + 5 * i;
        n += o[0]; sx += o[1]; sv += o[2];
        mx = std::max(mx, o[3]); mv = std::max(mv, o[4]);
    }
    const double cnt = n * (double)n_steps;
    out4[0] = std::sqrt(sx / cnt) * P.coord_to_x;
    out4[1] = std::sqrt(sv / cnt);
    out4[2] = mx * P.coord_to_x;
    out4[3] = mv;
    return SDE_OK;
}

int sde_reduce_f64(sde_ctx* c, const double* vals, uint64_t n, double* out3)
{
    if (!c || (!vals && n) || !out3) return SDE_EINVAL;
    if (n > 0xFFFFFFFFull * 32ull) return fail(c, SDE_EINVAL, "n too large");
    const uint64_t items = (n + 31ull) / 32ull;
    const Layout L = layout(1, items, 0);
    int rc;
    if ((rc = ensure_ws(c, L.total))) return rc;
    if ((rc = ensure_host(c, 64))) return rc;
    ++c->ws_gen;
    char* base = (char*)c->ws;
    double* partials = (double*)(base + L.off_partials);
    uint2* ranges = (uint2*)(base + L.off_ranges);
    double* out5 = (double*)(base + L.off_out5);
    const uint2 r0 = make_uint2(0u, (uint32_t)items);
    SDE_CUDA(c, cudaMemcpyAsync(ranges, &r0, sizeof(r0), cudaMemcpyHostToDevice, c->stream));
    SDE_CUDA(c, launch_reduce_items(vals, n, partials, c->stream));
    SDE_CUDA(c, launch_fold(partials, ranges, 1, out5, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(c->host, out5, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SDE_CUDA(c, cudaStreamSynchronize(c->stream));
    out3[0] = c->host[0];
    out3[1] = c->host[1];
    out3[2] = c->host[2];
    return SDE_OK;
}

int sde_philox_words(sde_ctx* c, const uint32_t* ctr, uint64_t n, uint64_t seed, uint32_t* out)
{
    if (!c || (!ctr && n) || (!out && n)) return SDE_EINVAL;
    if (n == 0) return SDE_OK;
    if (n > (1ull << 26)) return fail(c, SDE_EINVAL, "n too large");
    const size_t bytes = align256(16 * n);
    int rc;
    if ((rc = ensure_ws(c, 2 * bytes))) return rc;
    ++c->ws_gen;
    uint4* d_in = (uint4*)c->ws;
    uint4* d_out = (uint4*)((char*)c->ws + bytes);
    SDE_CUDA(c, cudaMemcpyAsync(d_in, ctr, 16 * n, cudaMemcpyHostToDevice, c->stream));
    const LaunchConsts K = make_launch(seed, 0, 0);
    SDE_CUDA(c, launch_philox(d_in, n, K, d_out, c->stream));
    SDE_CUDA(c, cudaMemcpyAsync(out, d_out, 16 * n, cudaMemcpyDeviceToHost, c->stream));
    SDE_CUDA(c, cudaStreamSynchronize(c->stream));
    return SDE_OK;
}

void sde_destroy(sde_ctx* c)
{
    if (!c) return;
    if (c->stream || c->own_stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->ws) cudaFree(c->ws);
    if (c->state) cudaFree(c->state);
    if (c->run_state) cudaFree(c->run_state);
    if (c->host) cudaFreeHost(c->host);
    if (c->done) cudaEventDestroy(c->done);
    for (cudaStream_t st : c->fan) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : c->fan_ev) cudaEventDestroy(ev);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
