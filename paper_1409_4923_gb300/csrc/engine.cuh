// engine.cuh -- device code of the Brownian-motor Monte Carlo engine (sm_103a).
//
// One GPU lane integrates one path (Algorithm 5 of the paper: the path state
// lives in registers for the whole run).  Paths are grouped in 32-path warp
// items pulled from a work counter, so a warp never waits for another warp and
// the ensemble reduction (Eq. 31) is a warp-shuffle tree per item plus a
// fixed-order FP64 fold per parameter point.
//
// Arithmetic: the path state and the step arithmetic are FP32 (Sec. 5,
// "use single precision ... folding of x"); the per-path window accumulators
// and every ensemble sum are FP64; the phase of the periodic drive is a 64-bit
// fixed-point fraction of a period, so it wraps modulo 2 pi exactly.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sde {

enum : uint32_t { kTagInit = 0u, kTagGauss = 1u, kTagPois = 2u, kTagDich = 3u };
enum { kModelInertial = 0, kModelOverdampedWashboard = 1, kModelPWL = 2 };
enum { kGauss3Point = 1, kGaussNormal = 2 };
enum : int32_t { kStatusOk = 0, kStatusTimedOut = -4 };

// ---------------------------------------------------------------- parameters

// Per-launch constants (kernel argument, read from the constant bank).
struct LaunchConsts {
    uint32_t rk0[10], rk1[10];   // Philox round keys: seed + r * Weyl constant
    uint32_t n_items;            // warp items in the launch
    uint64_t budget_ns;          // device-time budget per warp (from its start), 0 = none
};

// Per-point constants, precomputed on the host in FP64 and rounded once.
struct PointConsts {
    // integrator (coordinate units of the model; see the host code)
    float gdt;        // gamma dt                                 (inertial)
    float fdt;        // force amplitude x dt in coordinate units
    float wdt;        // coordinate advance per unit velocity per step (inertial)
    float whdt;       // half of wdt                              (inertial)
    float a_dt, F_dt; // drive amplitude and bias x dt in coordinate units
    uint64_t phase_step;  // omega dt / 2 pi as a 0.64 fixed-point fraction
    // noise
    float xi_c;       // Gaussian increment scale (G sqrt(3 dt) or G sqrt(dt))
    float aP_dt;      // Poisson bias a dt
    float zeta_l2;    // zeta ln 2 (amplitude from log2)
    float pois_cl2;   // ln 2 / (lambda dt)
    float Fb_dt, mFa_dt;        // dichotomous increments F_b dt and -F_a dt
    float mua_cl2, mub_cl2;     // ln 2 / (mu dt)
    double inv_lambda, inv_mua, inv_mub, dt64;   // exact (FP64) waiting times
    uint32_t d0_thresh;         // initial state F_b iff (w >> 8) < d0_thresh
    // initial state
    float x0_lo, x0_span, v0_lo, v0_span;
    // counters
    uint32_t c1_init, c1_gauss, c1_pois, c1_dich;   // (tag << 30) | point
    // run
    uint32_t n_tr, n_avg, n_paths;
    uint32_t path0;     // random-counter index of the run's first path (path ranges)
    double inv_window;  // 1 / (n_avg dt)
    double period;      // spatial period L in x units
    double coord_to_x;  // x = coordinate * coord_to_x (1 / 2 pi for washboards)
};

struct PathOutPtrs {
    double* X_f;
    float* v_f;
    double* vbar;
    uint32_t* jP;
    uint32_t* jD;
};

// ---------------------------------------------------------------- Philox

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;

// Philox4x32-10 (Salmon et al., SC'11) with precomputed round keys.
__device__ __forceinline__ uint4 philox10(uint4 c, const LaunchConsts& K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.rk0[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ K.rk1[r], (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ uint4 stream(const LaunchConsts& K, uint32_t c1, uint32_t path, uint32_t idx)
{
    return philox10(make_uint4(idx, c1, path, 0u), K);
}

// SFU approximations (PTX cos.approx / lg2.approx, flush-to-zero: the
// arguments here are never subnormal).
__device__ __forceinline__ float cos_sfu(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_sfu(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// phi = (w >> 8) 2^-24 in [0,1) and u = 1 - phi in (0,1], both exact in FP32.
__device__ __forceinline__ float phi24(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }
__device__ __forceinline__ float u24(uint32_t w) { return (float)(0x1000000u - (w >> 8)) * 0x1p-24f; }

// Waiting steps floor(-ln(u) / (rate dt)) (Algorithms 3 and 4).  The fast
// path uses the SFU log2 (absolute error about 2^-22 on u in (0, 1]); when
// the quotient lies within a margin of an integer that is 2^6 times the
// resulting error bound plus the rounding of the product, the decision is
// taken again with the paper's expression in FP64, so the integer equals the
// FP64 floor.
__device__ __forceinline__ int32_t wait_steps(uint32_t w, float cl2, double inv_rate, double dt)
{
    const float u = u24(w);
    float y = -lg2_sfu(u) * cl2;
    y = fminf(y, 1.0e9f);
    const float fl = floorf(y);
    const float fr = y - fl;
    const float m = __fmul_rn(cl2 + y, 0x1p-16f);
    if (fr < m || fr > 1.0f - m) {
        const double q = -inv_rate * log((double)u) / dt;
        return (int32_t)fmin(floor(q), 1.0e9);
    }
    return (int32_t)fl;
}

// Drive a cos(omega t_n) + F at step n, times dt in coordinate units.  The
// phase n omega dt / 2 pi is exact modulo one period in 64-bit fixed point;
// its top 32 bits give an angle in [-pi, pi) for the SFU cosine.
__device__ __forceinline__ float drive_at(uint32_t n, const PointConsts& P)
{
    const uint64_t ph = (uint64_t)n * P.phase_step;       // fraction of a period, mod 1
    const int32_t hi = (int32_t)(uint32_t)(ph >> 32);     // in [-1/2, 1/2) periods, Q0.32
    const float ang = (float)hi * 1.4629180792671596e-09f;   // 2 pi / 2^32
    return fmaf(P.a_dt, cos_sfu(ang), P.F_dt);
}

// ---------------------------------------------------------------- path state

// A jump process is held as its next event: the absolute step e at which it
// happens, its index J (events are numbered 1, 2, ...; index 0 is the initial
// countdown of Algorithms 3 and 4) and the cached words of the Philox block
// that serves the following events.  Algorithm 3's countdown s is e - n.
struct PathState {
    float c;      // folded coordinate: 2 pi x near [-pi, pi) (washboards), x in [-1, 1) (PWL)
    float v;      // velocity (inertial)
    float kf;     // whole periods folded out of c (exact integer in FP32)
    float c_i, kf_i;                // snapshot at t_i
    float sv, sv2;                  // FP32 window partials of v and v^2
    double svd, sv2d;               // FP64 window accumulators
    uint32_t eP, JP, pw2, pw3;                  // Poisson (Algorithm 3)
    uint32_t eD, JD, dst, dw1, dw2, dw3;        // dichotomous (Algorithm 4), dst 1 = F_b
};

template <int MODEL>
__device__ __forceinline__ void fold(PathState& S)
{
    if (MODEL == kModelPWL) {
        const float r = floorf((S.c + 1.0f) * 0.5f);     // c -> [-1, 1), period 2
        S.c = fmaf(-2.0f, r, S.c);
        S.kf += r;
    } else {
        const float r = rintf(S.c * 0.15915494309189535f); // c -> [-pi, pi]
        S.c = fmaf(-6.2831853071795865f, r, S.c);
        S.kf += r;
    }
}

// The inertial coordinate moves by at most 2 pi |v| dt per step, so folding it
// once per 4 steps keeps it inside (-4, 4), the same FP32 binade as [-pi, pi];
// the overdamped coordinates are folded every step.
template <int MODEL> struct FoldPerStep { static constexpr bool value = MODEL != kModelInertial; };

// base + (-V'(coordinate) x dt) in coordinate units.  Every multiply-add of
// the path is written out (fmaf, or a rounded product __fmul_rn / __dmul_rn
// where no fusion is wanted), so that the compiler's contraction choices
// cannot differ between the kernels that share this code (one or two paths
// per lane, segments, scans) and their results stay bit-identical.
template <int MODEL>
__device__ __forceinline__ float add_force_dt(float base, float c, const PointConsts& P)
{
    if (MODEL == kModelPWL) {
        // V' = +1 on [-1, 0), -1 on [0, 1) (mod 2): force -V0 V'
        const float y = fmaf(-2.0f, floorf(__fmul_rn(c + 1.0f, 0.5f)), c);
        return base + (y < 0.0f ? -P.fdt : P.fdt);
    } else {
        return fmaf(-P.fdt, cos_sfu(c), base);
    }
}

template <bool ACC>
__device__ __forceinline__ void accumulate(PathState& S)
{
    if (ACC) {
        S.sv += S.v;
        S.sv2 = fmaf(S.v, S.v, S.sv2);
    }
}

// h1 plus the corrector's jump increments: the Poissonian pj, and the
// dichotomous dg unless it is part of the drift (DICH == 2).
template <bool POIS, int DICH>
__device__ __forceinline__ float with_jumps(float h1, float pj, float dg)
{
    if (DICH == 1) return POIS ? h1 + (pj + dg) : h1 + dg;
    return POIS ? h1 + pj : h1;
}

// One step of Algorithm 1.  dxi: Gaussian increment; pj: Poissonian
// increment; dg: dichotomous increment Gamma_n dt; d0 / d1: drive x dt at
// t_n, t_{n+1}.  The jump increments enter the corrector only (Algorithm 1);
// with DICH == 2 the dichotomous force is instead a drift term, constant over
// the step, in all three drift evaluations.
// With CHI, chi receives Sec. 4's local-error indicator of the step, the
// predictor minus the corrector without the jump increments: chi[0] in the
// coordinate (whdt (v_Euler - v_predictor) = whdt (b1 - b2) / 2 inertial,
// (b2 - b3) / 2 overdamped), chi[1] in v ((b2 - b3) / 2, inertial).
template <int MODEL, bool POIS, int DICH, bool ACC, bool FOLD, bool CHI = false>
__device__ __forceinline__ void pc_step(PathState& S, const PointConsts& P, float dxi, float pj,
                                        float dg, float d0, float d1, float* chi = nullptr)
{
    if (DICH == 2) {
        d0 += dg;
        d1 += dg;
    }
    if (MODEL == kModelInertial) {
        const float b1 = add_force_dt<MODEL>(fmaf(-P.gdt, S.v, d0), S.c, P);   // F1_v dt
        const float vxi = S.v + dxi;
        float cb = fmaf(P.wdt, S.v, S.c);                                   // Euler x
        float vb = vxi + b1;                                                // Euler v
        const float b2 = add_force_dt<MODEL>(fmaf(-P.gdt, vb, d1), cb, P);
        const float ch = fmaf(P.whdt, S.v, S.c);
        const float h1 = fmaf(0.5f, b1, vxi);
        cb = fmaf(P.whdt, vb, ch);                                          // predictor x
        vb = fmaf(0.5f, b2, h1);                                            // predictor v
        const float b3 = add_force_dt<MODEL>(fmaf(-P.gdt, vb, d1), cb, P);
        S.c = fmaf(P.whdt, vb, ch);                                         // corrector x
        S.v = fmaf(0.5f, b3, with_jumps<POIS, DICH>(h1, pj, dg));           // corrector v
        accumulate<ACC>(S);
        if (CHI) {
            chi[0] = __fmul_rn(P.whdt, __fmul_rn(0.5f, b1 - b2));
            chi[1] = __fmul_rn(0.5f, b2 - b3);
        }
    } else {
        const float b1 = add_force_dt<MODEL>(d0, S.c, P);
        const float cxi = S.c + dxi;
        float cb = cxi + b1;                                                // Euler
        const float b2 = add_force_dt<MODEL>(d1, cb, P);
        const float h1 = fmaf(0.5f, b1, cxi);
        cb = fmaf(0.5f, b2, h1);                                            // predictor
        const float b3 = add_force_dt<MODEL>(d1, cb, P);
        S.c = fmaf(0.5f, b3, with_jumps<POIS, DICH>(h1, pj, dg));           // corrector
        if (CHI) {
            chi[0] = __fmul_rn(0.5f, b2 - b3);
            chi[1] = 0.0f;
        }
    }
    if (FOLD) fold<MODEL>(S);
}

// Algorithm 3 at event JP (step eP): the step's Poissonian increment z - a dt
// (scaled to coordinate units) and the step of the next event.
__device__ __forceinline__ float pois_event(PathState& S, const PointConsts& P,
                                            const LaunchConsts& K, uint32_t path)
{
    uint32_t wa, wb;
    if ((S.JP & 1u) == 0u) {
        const uint4 w = stream(K, P.c1_pois, path, S.JP >> 1);
        wa = w.x; wb = w.y; S.pw2 = w.z; S.pw3 = w.w;
    } else {
        wa = S.pw2; wb = S.pw3;
    }
    S.eP += (uint32_t)wait_steps(wa, P.pois_cl2, P.inv_lambda, P.dt64) + 1u;
    S.JP += 1u;
    return fmaf(-P.zeta_l2, lg2_sfu(u24(wb)), -P.aP_dt);
}

// Algorithm 4 at flip JD (step eD): the new state and the step of the next flip.
__device__ __forceinline__ void dich_event(PathState& S, const PointConsts& P,
                                           const LaunchConsts& K, uint32_t path)
{
    S.dst ^= 1u;
    const uint32_t k = S.JD & 3u;
    uint32_t w;
    if (k == 0u) {
        const uint4 b = stream(K, P.c1_dich, path, S.JD >> 2);
        w = b.x; S.dw1 = b.y; S.dw2 = b.z; S.dw3 = b.w;
    } else {
        w = k == 1u ? S.dw1 : (k == 2u ? S.dw2 : S.dw3);
    }
    const float cl2 = S.dst ? P.mub_cl2 : P.mua_cl2;
    const double inv_rate = S.dst ? P.inv_mub : P.inv_mua;
    S.eD += (uint32_t)wait_steps(w, cl2, inv_rate, P.dt64) + 1u;
    S.JD += 1u;
}

// Jump increments of step n with the events drawn as they happen.
template <bool POIS, int DICH>
__device__ __forceinline__ void jumps_inline(PathState& S, const PointConsts& P, const LaunchConsts& K,
                                             uint32_t path, uint32_t n, float& pj, float& dg)
{
    pj = 0.0f;
    dg = 0.0f;
    if (POIS) {
        pj = -P.aP_dt;
        if (n == S.eP) pj = pois_event(S, P, K, path);
    }
    if (DICH) {
        if (n == S.eD) dich_event(S, P, K, path);
        dg = S.dst ? P.Fb_dt : P.mFa_dt;
    }
}

// Events of the chunk [n0, n0 + 32), drawn before it is integrated so that
// the warp draws them together instead of one divergent branch per step.
// Bit i of pm marks a Poisson kick at step n0 + i, whose increments are
// queued in kick order in z0, z1, z2; bit i of dm is the dichotomous state at
// step n0 + i.  Returns false (and restores the Poisson state) when some lane
// of the warp has more than three kicks in the chunk: the warp then takes the
// Poisson events of this chunk inline.  All 32 lanes must call this together.
template <bool POIS, int DICH>
__device__ __forceinline__ bool chunk_events(PathState& S, const PointConsts& P, const LaunchConsts& K,
                                             uint32_t path, uint32_t n0, uint32_t& pm, float& z0,
                                             float& z1, float& z2, uint32_t& dm)
{
    bool fits = true;
    pm = 0u;
    z0 = z1 = z2 = 0.0f;
    dm = 0u;
    if (POIS) {
        const uint32_t e_save = S.eP, J_save = S.JP, w2_save = S.pw2, w3_save = S.pw3;
        uint32_t cnt = 0u;
        while (S.eP < n0 + 32u && cnt < 4u) {
            const uint32_t off = S.eP - n0;
            const float z = pois_event(S, P, K, path);
            pm |= 1u << off;
            z0 = cnt == 0u ? z : z0;
            z1 = cnt == 1u ? z : z1;
            z2 = cnt == 2u ? z : z2;
            ++cnt;
        }
        if (__any_sync(0xffffffffu, cnt > 3u)) {
            S.eP = e_save; S.JP = J_save; S.pw2 = w2_save; S.pw3 = w3_save;
            fits = false;
        }
    }
    if (DICH) {
        dm = S.dst ? 0xffffffffu : 0u;
        while (S.eD < n0 + 32u) {
            const uint32_t off = S.eD - n0;
            dich_event(S, P, K, path);
            dm ^= 0xffffffffu << off;
        }
    }
    return fits;
}

// Three-point increment (Algorithm 2, Eq. 25) from the running word r of the
// step (phi = r 2^-32), then r <- 6 r mod 2^32 for the next step that shares
// the word: the uniform of step 4i + k is frac(6^k phi_0).
__device__ __forceinline__ float three_point(uint32_t& r, const PointConsts& P)
{
    float d = r <= 1431655765u ? P.xi_c : 0.0f;        // phi <= 1/3
    d = r <= 715827882u ? -P.xi_c : d;                 // phi <= 1/6
    r *= 6u;
    return d;
}

// Gaussian increment for step 4 i + k from the word of its group (Box-Muller
// variant; the three-point law uses three_point).
template <int GAUSS>
__device__ __forceinline__ float gauss_inc(const uint4& w, uint32_t k, const PointConsts& P)
{
    if (GAUSS == kGaussNormal) {
        const uint32_t wa = k < 2u ? w.x : w.z;
        const uint32_t wb = k < 2u ? w.y : w.w;
        const float R = sqrtf(__fmul_rn(-2.0f, __logf(u24(wa))));
        // angle 2 pi phi - pi in [-pi, pi): cos/sin change sign
        const float T = fmaf(6.2831853071795865f, phi24(wb), -3.14159265358979f);
        float s, c;
        __sincosf(T, &s, &c);
        return __fmul_rn(__fmul_rn(-P.xi_c, R), (k & 1u) ? s : c);
    } else {
        return 0.0f;
    }
}

// Gaussian increment of step n drawn on its own (the chunked loops draw a
// block's word once for its 16 steps).
template <int GAUSS>
__device__ __forceinline__ float gauss_at(const PointConsts& P, const LaunchConsts& K, uint32_t path, uint32_t n)
{
    float dxi = 0.0f;
    if (GAUSS == kGauss3Point) {
        const uint4 w = stream(K, P.c1_gauss, path, n >> 4);
        const uint32_t q = (n >> 2) & 3u;
        uint32_t r = q == 0u ? w.x : (q == 1u ? w.y : (q == 2u ? w.z : w.w));
        const uint32_t k = n & 3u;
        r *= k == 0u ? 1u : (k == 1u ? 6u : (k == 2u ? 36u : 216u));
        dxi = three_point(r, P);
    } else if (GAUSS == kGaussNormal) {
        const uint4 w = stream(K, P.c1_gauss, path, n >> 2);
        dxi = gauss_inc<GAUSS>(w, n & 3u, P);
    }
    return dxi;
}

// Poissonian kicks drawn a window of chunks ahead, the counterpart of the
// dichotomous flip window below: per 32-step chunk a path has 0.41 kicks at
// lambda dt = 0.0128, but the warp's per-chunk event loop runs as often as its
// busiest lane needs.  Per window of kKickWinChunks chunks (512 steps) each
// lane draws its kicks once: bit i of mask word c marks a kick at step
// n0 + 32 c + i, and the kicks' increments (Algorithm 3: z - a dt) follow in
// kick order.  The queue holds kKickQueue increments; a lane whose queue fills
// up before the window's end shortens the window of the whole warp, which
// then draws its kicks again from the saved event state (the draws are a
// function of the event index, so the second pass gives the same kicks).  A
// chunk holds at most 32 kicks, so a window always keeps at least one chunk.
// The steps then pop the increments in order, with no per-chunk limit.
constexpr uint32_t kKickWinChunks = 16;
constexpr uint32_t kKickQueue = 32;
// Per lane: kKickWinChunks mask words, then kKickQueue + 1 increments (the
// last is read ahead after the final kick and never used), word-major with a
// stride of 32 so that each access is one word per lane.
constexpr uint32_t kKickWordsPerLane = kKickWinChunks + kKickQueue + 1u;
constexpr uint32_t kKickWordsPerWarp = kKickWordsPerLane * 32u;

// Kick windows run in the one-path-per-lane chunk loop of the point and scan
// kernels (not in segmented runs, whose saved state is the next event).
template <bool POIS, int GAUSS>
struct WindowedKicks { static constexpr bool value = POIS && GAUSS != kGaussNormal; };

// Two inertial paths per lane keep a kick window per path slot, each of
// kKick2Chunks chunks (256 steps) and a queue of kKick2Queue increments, so
// that a warp's two windows (6.4 KB) leave room for 24 warps per SM.  A queue
// this short does not guarantee that one chunk always fits: a warp in which
// some lane draws more kicks within the next chunk than its queue holds takes
// that chunk with the events drawn per chunk, as without windows (the same
// arithmetic).  At lambda dt = 0.1 a path has 3.2 kicks per chunk on average
// and more than 16 about once in 10^7 chunks.
constexpr uint32_t kKick2Chunks = 8;
constexpr uint32_t kKick2Queue = 16;
constexpr uint32_t kKick2WordsPerLane = kKick2Chunks + kKick2Queue + 1u;   // per path slot
constexpr uint32_t kKick2WordsPerWarp = 2u * kKick2WordsPerLane * 32u;

template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
struct WindowedKicks2 {
    static constexpr bool value = PPT == 2 && MODEL == kModelInertial && POIS && GAUSS != kGaussNormal;
};

// Kicks of one path in the steps [n0, wend) into the lane's words tw (stride
// 32): masks in words 0 .. kKickWinChunks - 1, increments from word
// kKickWinChunks.  Returns wend, or the step of the first kick not drawn when
// the queue filled up first; S then holds that kick as its next event.
// CH, QUEUE: the window's chunks and the queue's length (the two-path
// windows below are shorter).
template <uint32_t CH = kKickWinChunks, uint32_t QUEUE = kKickQueue>
__device__ __forceinline__ uint32_t window_kicks(PathState& S, const PointConsts& P, const LaunchConsts& K,
                                                 uint32_t path, uint32_t n0, uint32_t wend, uint32_t* tw)
{
#pragma unroll
    for (uint32_t c = 0; c < CH; ++c) tw[c * 32u] = 0u;
    float* tq = (float*)(tw + CH * 32u);
    uint32_t cnt = 0u;
    while (S.eP < wend && cnt < QUEUE) {
        const uint32_t off = S.eP - n0;
        tw[(off >> 5) * 32u] |= 1u << (off & 31u);
        tq[cnt * 32u] = pois_event(S, P, K, path);
        ++cnt;
    }
    return S.eP < wend ? S.eP : wend;
}

// Steps n in [n, n_end) one at a time (phase edges that are not whole
// 32-step chunks).
template <int MODEL, bool POIS, int DICH, int GAUSS, bool ACC>
__device__ __forceinline__ void single_steps(PathState& S, const PointConsts& P, const LaunchConsts& K,
                                             uint32_t path, uint32_t n, uint32_t n_end)
{
    for (; n < n_end; ++n) {
        const float dxi = gauss_at<GAUSS>(P, K, path, n);
        float pj, dg;
        jumps_inline<POIS, DICH>(S, P, K, path, n, pj, dg);
        pc_step<MODEL, POIS, DICH, ACC, true>(S, P, dxi, pj, dg, drive_at(n, P), drive_at(n + 1u, P));
    }
}

// One 32-step chunk from n0: 8 groups of 4 steps, the drive of step
// n0 + 1 + l in lane l (shuffled to every lane per step), jump events from
// the chunk masks (FAST) or inline.  Gaussian words: the three-point law
// takes one Philox call per 16-step block (one word per group of 4 steps),
// the Box-Muller variant one per group.  w holds the words of the chunk's
// first block (group); each block (group) draws the next one's words while it
// integrates, so the Philox multiplies interleave with the step arithmetic,
// and w returns holding those that follow the chunk.
// With QUEUE the kick increments come from the lane's window queue (stride
// 32 words): *qp points at the entry held in *zq, the next kick's increment;
// each kick advances *qp by one entry and loads the following one.
template <int MODEL, bool POIS, int DICH, int GAUSS, bool ACC, bool FAST, bool QUEUE = false>
__device__ __forceinline__ void chunk_steps(PathState& S, const PointConsts& P, const LaunchConsts& K,
                                            uint32_t path, uint32_t n0, float dch, float& dcur,
                                            uint4& w, uint32_t pm, float z0, float z1, float z2,
                                            uint32_t dm, const float** qp = nullptr,
                                            float* zq = nullptr)
{
    // Without Box-Muller words the chunk is two 16-step blocks of one Philox
    // call each: the block's four groups are unrolled, so each group's word
    // and each step's event bit are compile-time selections.  The rare chunks
    // whose Poisson events take the inline path keep the compact loop of one
    // group per iteration below.
    constexpr bool kBlockLoop = GAUSS != kGaussNormal && (!POIS || FAST || QUEUE);
    if (kBlockLoop) {
#pragma unroll 1
        for (uint32_t b = 0; b < 2u; ++b) {
            uint4 wn = make_uint4(0u, 0u, 0u, 0u);
            if (GAUSS == kGauss3Point) wn = stream(K, P.c1_gauss, path, (n0 >> 4) + b + 1u);
#pragma unroll
            for (uint32_t q = 0; q < 4u; ++q) {
                uint32_t r = q == 0u ? w.x : (q == 1u ? w.y : (q == 2u ? w.z : w.w));
#pragma unroll
                for (uint32_t k = 0; k < 4u; ++k) {
                    const float dnext = __shfl_sync(0xffffffffu, dch, (int)(q * 4u + k));
                    const float dxi = GAUSS == kGauss3Point ? three_point(r, P) : 0.0f;
                    float pj = 0.0f, dg = 0.0f;
                    if (POIS && QUEUE) {
                        const bool kick = (pm & (1u << (q * 4u + k))) != 0u;
                        pj = kick ? *zq : -P.aP_dt;
                        if (kick) {
                            *qp += 32;
                            *zq = **qp;
                        }
                    } else if (POIS) {
                        const bool kick = (pm & (1u << (q * 4u + k))) != 0u;
                        pj = kick ? z0 : -P.aP_dt;
                        z0 = kick ? z1 : z0;
                        z1 = kick ? z2 : z1;
                    }
                    if (DICH) dg = (dm & (1u << (q * 4u + k))) != 0u ? P.Fb_dt : P.mFa_dt;
                    pc_step<MODEL, POIS, DICH, ACC, FoldPerStep<MODEL>::value>(S, P, dxi, pj, dg, dcur,
                                                                               dnext);
                    dcur = dnext;
                }
                if (!FoldPerStep<MODEL>::value) fold<MODEL>(S);
            }
            w = wn;
            pm >>= 16;
            dm >>= 16;
            dch = __shfl_down_sync(0xffffffffu, dch, 16);   // the second block's drive values
        }
        return;
    }
    constexpr int kGroupUnroll = POIS ? 1 : 2;
    uint4 wn = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll kGroupUnroll
    for (uint32_t g = 0; g < 8u; ++g) {
        uint32_t r = 0u;
        if (GAUSS == kGauss3Point) {
            if ((g & 3u) == 0u) wn = stream(K, P.c1_gauss, path, (n0 >> 4) + (g >> 2) + 1u);
            const uint32_t q = g & 3u;
            r = q == 0u ? w.x : (q == 1u ? w.y : (q == 2u ? w.z : w.w));
        } else if (GAUSS == kGaussNormal) {
            wn = stream(K, P.c1_gauss, path, (n0 >> 2) + g + 1u);
        }
#pragma unroll
        for (uint32_t k = 0; k < 4u; ++k) {
            const float dnext = __shfl_sync(0xffffffffu, dch, (int)(g * 4u + k));
            float dxi = 0.0f;
            if (GAUSS == kGauss3Point) dxi = three_point(r, P);
            else if (GAUSS == kGaussNormal) dxi = gauss_inc<GAUSS>(w, k, P);
            float pj = 0.0f, dg = 0.0f;
            if (POIS) {
                if (FAST) {
                    const bool kick = (pm & (1u << k)) != 0u;
                    pj = kick ? z0 : -P.aP_dt;
                    z0 = kick ? z1 : z0;
                    z1 = kick ? z2 : z1;
                } else {
                    pj = -P.aP_dt;
                    if (n0 + g * 4u + k == S.eP) pj = pois_event(S, P, K, path);
                }
            }
            if (DICH) dg = (dm & (1u << k)) != 0u ? P.Fb_dt : P.mFa_dt;
            pc_step<MODEL, POIS, DICH, ACC, FoldPerStep<MODEL>::value>(S, P, dxi, pj, dg, dcur, dnext);
            dcur = dnext;
        }
        if (GAUSS == kGaussNormal || (GAUSS == kGauss3Point && (g & 3u) == 3u)) w = wn;
        pm >>= 4;
        dm >>= 4;
        if (!FoldPerStep<MODEL>::value) fold<MODEL>(S);
    }
}

// Steps n in [n, n_end): edges one at a time, whole 32-step chunks with the
// events of each chunk drawn up front.  The FP32 window partials are moved to
// the FP64 accumulators whenever a chunk ends on a multiple of 256 steps.
// Chunks and flushes sit at absolute step positions, so a run cut into
// segments at multiples of 32 steps takes the same arithmetic as one launch.
// All 32 lanes of the warp must call this together.
// WIN: the Poissonian kicks are drawn in windows (WindowedKicks), in the
// lane's kKickWordsPerLane words of shared memory at win (stride 32).
template <int MODEL, bool POIS, int DICH, int GAUSS, bool ACC, bool WIN = false>
__device__ __forceinline__ void run_steps(PathState& S, const PointConsts& P, const LaunchConsts& K,
                                          uint32_t path, uint32_t lane, uint32_t n, uint32_t n_end,
                                          uint32_t* win = nullptr)
{
    uint32_t head = n;                                   // first chunk boundary
    if ((n & 31u) != 0u) head = min(n_end, (n + 31u) & ~31u);
    if (head > n) {
        single_steps<MODEL, POIS, DICH, GAUSS, ACC>(S, P, K, path, n, head);
        n = head;
    }
    if (n + 32u <= n_end) {
        float dcur = drive_at(n, P);
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (GAUSS == kGauss3Point) w = stream(K, P.c1_gauss, path, n >> 4);
        else if (GAUSS == kGaussNormal) w = stream(K, P.c1_gauss, path, n >> 2);
        if constexpr (WIN && WindowedKicks<POIS, GAUSS>::value) {
            uint32_t* tw = win;
            const float* tq = (const float*)(win + kKickWinChunks * 32u);
            while (n + 32u <= n_end) {
                uint32_t wend = n + 32u * min(kKickWinChunks, (n_end - n) >> 5);
                const uint32_t e_s = S.eP, j_s = S.JP, w2_s = S.pw2, w3_s = S.pw3;
                const uint32_t cover = __reduce_min_sync(0xffffffffu, window_kicks(S, P, K, path, n, wend, tw));
                if (cover < wend) {
                    // a lane's queue filled up: the warp's window ends at the last
                    // whole chunk that every lane covers (at least one), drawn again
                    wend = n + ((cover - n) & ~31u);
                    S.eP = e_s; S.JP = j_s; S.pw2 = w2_s; S.pw3 = w3_s;
                    window_kicks(S, P, K, path, n, wend, tw);
                }
                const float* qp = tq;
                float zq = tq[0];
#pragma unroll 1
                for (const uint32_t* pmw = tw; n < wend; n += 32u, pmw += 32) {
                    const float dch = drive_at(n + 1u + lane, P);
                    uint32_t pm_unused, dm;
                    float z0, z1, z2;
                    chunk_events<false, DICH>(S, P, K, path, n, pm_unused, z0, z1, z2, dm);
                    chunk_steps<MODEL, POIS, DICH, GAUSS, ACC, true, true>(S, P, K, path, n, dch, dcur, w,
                                                                           *pmw, z0, z1, z2, dm, &qp,
                                                                           &zq);
                    if (ACC && ((n + 32u) & 255u) == 0u) {
                        S.svd += (double)S.sv;
                        S.sv2d += (double)S.sv2;
                        S.sv = 0.0f;
                        S.sv2 = 0.0f;
                    }
                }
            }
        } else
        for (; n + 32u <= n_end; n += 32u) {
            const float dch = drive_at(n + 1u + lane, P);
            uint32_t pm, dm;
            float z0, z1, z2;
            if (chunk_events<POIS, DICH>(S, P, K, path, n, pm, z0, z1, z2, dm))
                chunk_steps<MODEL, POIS, DICH, GAUSS, ACC, true>(S, P, K, path, n, dch, dcur, w, pm,
                                                                 z0, z1, z2, dm);
            else
                chunk_steps<MODEL, POIS, DICH, GAUSS, ACC, false>(S, P, K, path, n, dch, dcur, w, pm,
                                                                  z0, z1, z2, dm);
            if (ACC && ((n + 32u) & 255u) == 0u) {
                S.svd += (double)S.sv;
                S.sv2d += (double)S.sv2;
                S.sv = 0.0f;
                S.sv2 = 0.0f;
            }
        }
    }
    if (n < n_end) single_steps<MODEL, POIS, DICH, GAUSS, ACC>(S, P, K, path, n, n_end);
}

template <int MODEL, bool POIS, int DICH>
__device__ __forceinline__ void init_path(PathState& S, const PointConsts& P, const LaunchConsts& K,
                                          uint32_t path)
{
    const uint4 w = stream(K, P.c1_init, path, 0u);
    const float x0 = fmaf(P.x0_span, phi24(w.x), P.x0_lo);
    S.c = MODEL == kModelPWL ? x0 : x0 * 6.2831853071795865f;
    S.v = MODEL == kModelInertial ? fmaf(P.v0_span, phi24(w.y), P.v0_lo) : 0.0f;
    S.kf = 0.0f;
    fold<MODEL>(S);
    S.sv = S.sv2 = 0.0f;
    S.svd = S.sv2d = 0.0;
    S.eP = 0xffffffffu; S.JP = 0u; S.pw2 = S.pw3 = 0u;
    S.eD = 0xffffffffu; S.JD = 0u; S.dst = 0u; S.dw1 = S.dw2 = S.dw3 = 0u;
    if (POIS) {
        const uint4 e = stream(K, P.c1_pois, path, 0u);        // index 0: initial countdown
        S.eP = (uint32_t)wait_steps(e.x, P.pois_cl2, P.inv_lambda, P.dt64);
        S.JP = 1u;
        S.pw2 = e.z; S.pw3 = e.w;
    }
    if (DICH) {
        S.dst = (w.z >> 8) < P.d0_thresh ? 1u : 0u;             // stationary start
        const uint4 e = stream(K, P.c1_dich, path, 0u);
        S.eD = S.dst ? (uint32_t)wait_steps(e.x, P.mub_cl2, P.inv_mub, P.dt64)
                     : (uint32_t)wait_steps(e.x, P.mua_cl2, P.inv_mua, P.dt64);
        S.JD = 1u;
        S.dw1 = e.y; S.dw2 = e.z; S.dw3 = e.w;
    }
}

struct PathResult {
    double X_f, vbar, sum_v, sum_v2;
    float v_f;
    uint32_t jP, jD;
};

// Eq. 31 summand and the path's other results from its final state.
template <int MODEL, bool POIS, int DICH>
__device__ __forceinline__ void finish_path(const PathState& S, const PointConsts& P, PathResult& R)
{
    const double dX = __fma_rn((double)S.kf - (double)S.kf_i, P.period,
                               __dmul_rn((double)S.c - (double)S.c_i, P.coord_to_x));
    R.X_f = __fma_rn((double)S.kf, P.period, __dmul_rn((double)S.c, P.coord_to_x));
    R.vbar = __dmul_rn(dX, P.inv_window);
    R.sum_v = S.svd + (double)S.sv;
    R.sum_v2 = S.sv2d + (double)S.sv2;
    R.v_f = S.v;
    R.jP = POIS ? S.JP - 1u : 0u;     // index of the last event that happened
    R.jD = DICH ? S.JD - 1u : 0u;
}

// WIN: draw the Poissonian kicks in windows, in the lane's shared-memory
// words at win (see WindowedKicks).
template <int MODEL, bool POIS, int DICH, int GAUSS, bool WIN = false>
__device__ __forceinline__ void simulate_path(const PointConsts& P, const LaunchConsts& K,
                                              uint32_t path, uint32_t lane, PathResult& R,
                                              uint32_t* win = nullptr)
{
    PathState S;
    init_path<MODEL, POIS, DICH>(S, P, K, path);
    run_steps<MODEL, POIS, DICH, GAUSS, false, WIN>(S, P, K, path, lane, 0u, P.n_tr, win);
    if (!FoldPerStep<MODEL>::value) fold<MODEL>(S);
    S.c_i = S.c;
    S.kf_i = S.kf;
    run_steps<MODEL, POIS, DICH, GAUSS, MODEL == kModelInertial, WIN>(S, P, K, path, lane, P.n_tr,
                                                                      P.n_tr + P.n_avg, win);
    finish_path<MODEL, POIS, DICH>(S, P, R);
}

// Steps [na, nb) of a path whose state is at step na: the part of the
// transient in the segment, the snapshot at t_i if the transient ends in it,
// then the part of the averaging window.  Cut points at multiples of 32 steps
// (or at n_transient) give the arithmetic of simulate_path exactly.
template <int MODEL, bool POIS, int DICH, int GAUSS>
__device__ __forceinline__ void advance_path(PathState& S, const PointConsts& P, const LaunchConsts& K,
                                             uint32_t path, uint32_t lane, uint32_t na, uint32_t nb)
{
    const uint32_t ntr = P.n_tr;
    if (na < ntr) run_steps<MODEL, POIS, DICH, GAUSS, false>(S, P, K, path, lane, na, min(nb, ntr));
    if ((na < ntr && nb >= ntr) || (na == 0u && ntr == 0u)) {
        if (!FoldPerStep<MODEL>::value) fold<MODEL>(S);
        S.c_i = S.c;
        S.kf_i = S.kf;
    }
    if (nb > ntr)
        run_steps<MODEL, POIS, DICH, GAUSS, MODEL == kModelInertial>(S, P, K, path, lane,
                                                                     max(na, ntr), nb);
}

// ---------------------------------------------------------------- several paths per lane

// The same integration for PPT paths per lane, interleaved step by step so
// that their independent dependency chains fill each other's latencies; the
// drive values and the loop are shared.  Two inertial paths run their chunks
// on packed FP32 pairs (chunk_steps_x2).  Every path takes exactly the
// operations of run_steps (a chunk whose Poisson events do not fit the queue
// of some path takes all paths' events inline, which gives the same values),
// so results do not depend on PPT.

template <bool POIS, int DICH, int PPT>
__device__ __forceinline__ bool chunk_events_multi(PathState (&S)[PPT], const PointConsts& P,
                                                   const LaunchConsts& K, const uint32_t (&path)[PPT],
                                                   uint32_t n0, uint32_t (&pm)[PPT], float (&z0)[PPT],
                                                   float (&z1)[PPT], float (&z2)[PPT], uint32_t (&dm)[PPT])
{
    bool over = false;
    uint32_t e_save[PPT], J_save[PPT], w2_save[PPT], w3_save[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        pm[p] = 0u;
        z0[p] = z1[p] = z2[p] = 0.0f;
        dm[p] = 0u;
        if (POIS) {
            e_save[p] = S[p].eP; J_save[p] = S[p].JP; w2_save[p] = S[p].pw2; w3_save[p] = S[p].pw3;
            uint32_t cnt = 0u;
            while (S[p].eP < n0 + 32u && cnt < 4u) {
                const uint32_t off = S[p].eP - n0;
                const float z = pois_event(S[p], P, K, path[p]);
                pm[p] |= 1u << off;
                z0[p] = cnt == 0u ? z : z0[p];
                z1[p] = cnt == 1u ? z : z1[p];
                z2[p] = cnt == 2u ? z : z2[p];
                ++cnt;
            }
            over |= cnt > 3u;
        }
        if (DICH) {
            dm[p] = S[p].dst ? 0xffffffffu : 0u;
            while (S[p].eD < n0 + 32u) {
                const uint32_t off = S[p].eD - n0;
                dich_event(S[p], P, K, path[p]);
                dm[p] ^= 0xffffffffu << off;
            }
        }
    }
    if (POIS && __any_sync(0xffffffffu, over)) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            S[p].eP = e_save[p]; S[p].JP = J_save[p]; S[p].pw2 = w2_save[p]; S[p].pw3 = w3_save[p];
        }
        return false;
    }
    return true;
}

// Two inertial paths per lane on the packed FP32 pair instructions of sm_100
// and later (__ffma2_rn, __fadd2_rn, __fmul2_rn: per component exactly
// __fmaf_rn, __fadd_rn, __fmul_rn).  Component x is path 0, y path 1; every
// operation of pc_step, fold and accumulate is applied to the pair in the same
// order, so each path takes the arithmetic of one path per lane bit for bit,
// while the step issues about half as many FP32 instructions.  The SFU
// cosines, the three-point draws and the jump selections stay per path.  The
// chunk is two 16-step blocks as in chunk_steps.
__device__ __forceinline__ float2 cos2_sfu(float2 x) { return make_float2(cos_sfu(x.x), cos_sfu(x.y)); }

template <bool POIS, int DICH>
__device__ __forceinline__ float2 with_jumps2(float2 h1, float2 pj, float2 dg)
{
    if (DICH == 1) return POIS ? __fadd2_rn(h1, __fadd2_rn(pj, dg)) : __fadd2_rn(h1, dg);
    return POIS ? __fadd2_rn(h1, pj) : h1;
}

// QUEUE: the kick increments come from the two path slots' window queues
// (stride 32 words): qp[p] points at the entry held in zq[p], the slot's next
// kick's increment.
template <bool POIS, int DICH, int GAUSS, bool ACC, bool QUEUE = false>
__device__ __forceinline__ void chunk_steps_x2(PathState (&S)[2], const PointConsts& P,
                                               const LaunchConsts& K, const uint32_t (&path)[2],
                                               uint32_t n0, float dch, float& dcur, uint4 (&w)[2],
                                               uint32_t (&pm)[2], float (&z0)[2], float (&z1)[2],
                                               float (&z2)[2], uint32_t (&dm)[2],
                                               const float** qp = nullptr, float* zq = nullptr)
{
    const float2 ngdt = make_float2(-P.gdt, -P.gdt), nfdt = make_float2(-P.fdt, -P.fdt);
    const float2 wdt = make_float2(P.wdt, P.wdt), whdt = make_float2(P.whdt, P.whdt);
    const float2 half = make_float2(0.5f, 0.5f);
    float2 c = make_float2(S[0].c, S[1].c), v = make_float2(S[0].v, S[1].v);
    float2 kf = make_float2(S[0].kf, S[1].kf);
    float2 sv = make_float2(S[0].sv, S[1].sv), sv2 = make_float2(S[0].sv2, S[1].sv2);
#pragma unroll 1
    for (uint32_t b = 0; b < 2u; ++b) {
        uint4 wn[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            wn[p] = make_uint4(0u, 0u, 0u, 0u);
            if (GAUSS == kGauss3Point) wn[p] = stream(K, P.c1_gauss, path[p], (n0 >> 4) + b + 1u);
        }
        // With Poisson noise the block keeps one 4-step group per iteration:
        // the two paths' kick queues unrolled over 16 steps overflow the
        // instruction cache (measured: half speed, "no instruction" stalls).
#pragma unroll ((POIS && !QUEUE) ? 1 : 4)
        for (uint32_t q = 0; q < 4u; ++q) {
            uint32_t r[2];
#pragma unroll
            for (int p = 0; p < 2; ++p)
                r[p] = q == 0u ? w[p].x : (q == 1u ? w[p].y : (q == 2u ? w[p].z : w[p].w));
#pragma unroll
            for (uint32_t k = 0; k < 4u; ++k) {
                const float dnext = __shfl_sync(0xffffffffu, dch, (int)(q * 4u + k));
                const uint32_t bit = 1u << (q * 4u + k);
                float2 dxi = make_float2(0.0f, 0.0f), pj = dxi, dg = dxi;
                if (GAUSS == kGauss3Point) {
                    dxi.x = three_point(r[0], P);
                    dxi.y = three_point(r[1], P);
                }
                if (POIS && QUEUE) {
                    float pv[2];
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const bool kick = (pm[p] & bit) != 0u;
                        pv[p] = kick ? zq[p] : -P.aP_dt;
                        if (kick) {
                            qp[p] += 32;
                            zq[p] = *qp[p];
                        }
                    }
                    pj = make_float2(pv[0], pv[1]);
                } else if (POIS) {
                    float pv[2];
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const bool kick = (pm[p] & bit) != 0u;
                        pv[p] = kick ? z0[p] : -P.aP_dt;
                        z0[p] = kick ? z1[p] : z0[p];
                        z1[p] = kick ? z2[p] : z1[p];
                    }
                    pj = make_float2(pv[0], pv[1]);
                }
                if (DICH) {
                    dg.x = (dm[0] & bit) != 0u ? P.Fb_dt : P.mFa_dt;
                    dg.y = (dm[1] & bit) != 0u ? P.Fb_dt : P.mFa_dt;
                }
                float2 d0 = make_float2(dcur, dcur), d1 = make_float2(dnext, dnext);
                if (DICH == 2) {
                    d0 = __fadd2_rn(d0, dg);
                    d1 = __fadd2_rn(d1, dg);
                }
                // Algorithm 1 on (x, v), as pc_step
                const float2 b1 = __ffma2_rn(nfdt, cos2_sfu(c), __ffma2_rn(ngdt, v, d0));
                const float2 vxi = __fadd2_rn(v, dxi);
                float2 cb = __ffma2_rn(wdt, v, c);
                float2 vb = __fadd2_rn(vxi, b1);
                const float2 b2 = __ffma2_rn(nfdt, cos2_sfu(cb), __ffma2_rn(ngdt, vb, d1));
                const float2 ch = __ffma2_rn(whdt, v, c);
                const float2 h1 = __ffma2_rn(half, b1, vxi);
                cb = __ffma2_rn(whdt, vb, ch);
                vb = __ffma2_rn(half, b2, h1);
                const float2 b3 = __ffma2_rn(nfdt, cos2_sfu(cb), __ffma2_rn(ngdt, vb, d1));
                c = __ffma2_rn(whdt, vb, ch);
                v = __ffma2_rn(half, b3, with_jumps2<POIS, DICH>(h1, pj, dg));
                if (ACC) {
                    sv = __fadd2_rn(sv, v);
                    sv2 = __ffma2_rn(v, v, sv2);
                }
                dcur = dnext;
            }
            // fold, as fold<kModelInertial>
            const float2 t = __fmul2_rn(c, make_float2(0.15915494309189535f, 0.15915494309189535f));
            const float2 rr = make_float2(rintf(t.x), rintf(t.y));
            c = __ffma2_rn(make_float2(-6.2831853071795865f, -6.2831853071795865f), rr, c);
            kf = __fadd2_rn(kf, rr);
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            w[p] = wn[p];
            pm[p] >>= 16;
            dm[p] >>= 16;
        }
        dch = __shfl_down_sync(0xffffffffu, dch, 16);   // the second block's drive values
    }
    S[0].c = c.x; S[1].c = c.y;
    S[0].v = v.x; S[1].v = v.y;
    S[0].kf = kf.x; S[1].kf = kf.y;
    S[0].sv = sv.x; S[1].sv = sv.y;
    S[0].sv2 = sv2.x; S[1].sv2 = sv2.y;
}

// Dichotomous flips drawn a window of chunks ahead.  Per 32-step chunk a
// path has 0.41 flips on average at the 2^20-path workload's rates
// (1 - e^{-mu dt} = 0.0127 per step), but the warp's event loop runs as often
// as its busiest lane needs: about 2.1 times per chunk and path slot.  Drawn
// for kWinChunks = 32 chunks (1024 steps, 13 flips per path on average) at
// once, the loop runs about 21 times per window instead of 67, with more
// lanes busy in each pass, and every chunk then reads its state mask from
// shared memory.  The flips are those of Algorithm 4 (the same countdowns,
// evaluated earlier), so the results do not change.  Measured on that
// workload (2^20 paths x 440,000 steps): 504 ms against 574 ms with the flips
// drawn per chunk, and 541 ms with windows of 16 chunks.  The window takes
// 8 KB of shared memory per warp (192 KB per SM at 24 warps).
constexpr uint32_t kWinChunks = 32;

template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
struct WindowedFlips {
    static constexpr bool value = PPT == 2 && MODEL == kModelInertial && !POIS && DICH != 0 &&
                                  GAUSS != kGaussNormal;
};

// Shared-memory words of one warp's flip window: kWinChunks words per path
// slot and lane, stored word-major so that each access is one word per lane
// (conflict-free).
constexpr uint32_t kWinWordsPerWarp = 2u * kWinChunks * 32u;

// Flips of one path in the steps [n0, n0 + 32 nch) (nch <= kWinChunks):
// word c of tw (stride 32) receives chunk c's state mask, bit i the
// dichotomous state at step n0 + 32 c + i, as chunk_events builds it.  First
// each flip at step n0 + o toggles the bits from o to the end of its word,
// then a pass carries each word's last state into the next.  On return S
// holds the first flip at or after the window's end.  A thread reads back
// only its own words.
__device__ __forceinline__ void window_flips(PathState& S, const PointConsts& P, const LaunchConsts& K,
                                             uint32_t path, uint32_t n0, uint32_t nch, uint32_t* tw)
{
    uint32_t carry = S.dst ? 0xffffffffu : 0u;     // state before the window
#pragma unroll
    for (uint32_t c = 0; c < kWinChunks; ++c) tw[c * 32u] = 0u;
    const uint32_t wend = n0 + 32u * nch;
    while (S.eD < wend) {
        const uint32_t off = S.eD - n0;
        tw[(off >> 5) * 32u] ^= 0xffffffffu << (off & 31u);
        dich_event(S, P, K, path);
    }
#pragma unroll
    for (uint32_t c = 0; c < kWinChunks; ++c) {
        const uint32_t m = tw[c * 32u] ^ carry;
        tw[c * 32u] = m;
        carry = (uint32_t)((int32_t)m >> 31);
    }
}

template <int MODEL, bool POIS, int DICH, int GAUSS, bool ACC, bool FAST, int PPT>
__device__ __forceinline__ void chunk_steps_multi(PathState (&S)[PPT], const PointConsts& P,
                                                  const LaunchConsts& K, const uint32_t (&path)[PPT],
                                                  uint32_t n0, float dch, float& dcur, uint4 (&w)[PPT],
                                                  uint32_t (&pm)[PPT], float (&z0)[PPT], float (&z1)[PPT],
                                                  float (&z2)[PPT], uint32_t (&dm)[PPT])
{
    if constexpr (PPT == 2 && MODEL == kModelInertial && GAUSS != kGaussNormal && (!POIS || FAST)) {
        chunk_steps_x2<POIS, DICH, GAUSS, ACC>(S, P, K, path, n0, dch, dcur, w, pm, z0, z1, z2, dm);
        return;
    }
    uint4 wn[PPT];
#pragma unroll 1
    for (uint32_t g = 0; g < 8u; ++g) {
        uint32_t r[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            r[p] = 0u;
            if (GAUSS == kGauss3Point) {
                if ((g & 3u) == 0u) wn[p] = stream(K, P.c1_gauss, path[p], (n0 >> 4) + (g >> 2) + 1u);
                const uint32_t q = g & 3u;
                r[p] = q == 0u ? w[p].x : (q == 1u ? w[p].y : (q == 2u ? w[p].z : w[p].w));
            } else if (GAUSS == kGaussNormal) {
                wn[p] = stream(K, P.c1_gauss, path[p], (n0 >> 2) + g + 1u);
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < 4u; ++k) {
            const float dnext = __shfl_sync(0xffffffffu, dch, (int)(g * 4u + k));
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                float dxi = 0.0f;
                if (GAUSS == kGauss3Point) dxi = three_point(r[p], P);
                else if (GAUSS == kGaussNormal) dxi = gauss_inc<GAUSS>(w[p], k, P);
                float pj = 0.0f, dg = 0.0f;
                if (POIS) {
                    if (FAST) {
                        const bool kick = (pm[p] & (1u << k)) != 0u;
                        pj = kick ? z0[p] : -P.aP_dt;
                        z0[p] = kick ? z1[p] : z0[p];
                        z1[p] = kick ? z2[p] : z1[p];
                    } else {
                        pj = -P.aP_dt;
                        if (n0 + g * 4u + k == S[p].eP) pj = pois_event(S[p], P, K, path[p]);
                    }
                }
                if (DICH) dg = (dm[p] & (1u << k)) != 0u ? P.Fb_dt : P.mFa_dt;
                pc_step<MODEL, POIS, DICH, ACC, FoldPerStep<MODEL>::value>(S[p], P, dxi, pj, dg, dcur,
                                                                           dnext);
            }
            dcur = dnext;
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            if (GAUSS == kGaussNormal || (GAUSS == kGauss3Point && (g & 3u) == 3u)) w[p] = wn[p];
            pm[p] >>= 4;
            dm[p] >>= 4;
            if (!FoldPerStep<MODEL>::value) fold<MODEL>(S[p]);
        }
    }
}

// The FP32 window partials move to the FP64 accumulators when the chunk
// from n ends on a multiple of 256 steps.
template <bool ACC, int PPT>
__device__ __forceinline__ void flush_window_sums(PathState (&S)[PPT], uint32_t n)
{
    if (ACC && ((n + 32u) & 255u) == 0u) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            S[p].svd += (double)S[p].sv;
            S[p].sv2d += (double)S[p].sv2;
            S[p].sv = 0.0f;
            S[p].sv2 = 0.0f;
        }
    }
}

// The chunk from n with its events drawn before it (chunk_events_multi),
// then the window flush.
template <int MODEL, bool POIS, int DICH, int GAUSS, bool ACC, int PPT>
__device__ __forceinline__ void chunk_drawn_per_chunk(PathState (&S)[PPT], const PointConsts& P,
                                                      const LaunchConsts& K, const uint32_t (&path)[PPT],
                                                      uint32_t lane, uint32_t n, float& dcur, uint4 (&w)[PPT])
{
    const float dch = drive_at(n + 1u + lane, P);
    uint32_t pm[PPT], dm[PPT];
    float z0[PPT], z1[PPT], z2[PPT];
    if (chunk_events_multi<POIS, DICH, PPT>(S, P, K, path, n, pm, z0, z1, z2, dm))
        chunk_steps_multi<MODEL, POIS, DICH, GAUSS, ACC, true, PPT>(S, P, K, path, n, dch, dcur, w, pm, z0, z1,
                                                                    z2, dm);
    else
        chunk_steps_multi<MODEL, POIS, DICH, GAUSS, ACC, false, PPT>(S, P, K, path, n, dch, dcur, w, pm, z0, z1,
                                                                     z2, dm);
    flush_window_sums<ACC, PPT>(S, n);
}

template <int MODEL, bool POIS, int DICH, int GAUSS, bool ACC, int PPT>
__device__ __forceinline__ void run_steps_multi(PathState (&S)[PPT], const PointConsts& P,
                                                const LaunchConsts& K, const uint32_t (&path)[PPT],
                                                uint32_t lane, uint32_t n, uint32_t n_end,
                                                uint32_t* win = nullptr)
{
    uint32_t head = n;
    if ((n & 31u) != 0u) head = min(n_end, (n + 31u) & ~31u);
    if (head > n) {
#pragma unroll
        for (int p = 0; p < PPT; ++p)
            single_steps<MODEL, POIS, DICH, GAUSS, ACC>(S[p], P, K, path[p], n, head);
        n = head;
    }
    if (n + 32u <= n_end) {
        float dcur = drive_at(n, P);
        uint4 w[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            w[p] = make_uint4(0u, 0u, 0u, 0u);
            if (GAUSS == kGauss3Point) w[p] = stream(K, P.c1_gauss, path[p], n >> 4);
            else if (GAUSS == kGaussNormal) w[p] = stream(K, P.c1_gauss, path[p], n >> 2);
        }
        if constexpr (WindowedFlips<MODEL, POIS, DICH, GAUSS, PPT>::value) {
            // chunks in windows of kWinChunks, flips drawn at the start of each
            while (n + 32u <= n_end) {
                const uint32_t nch = min(kWinChunks, (n_end - n) >> 5);
                window_flips(S[0], P, K, path[0], n, nch, win + lane);
                window_flips(S[1], P, K, path[1], n, nch, win + kWinChunks * 32u + lane);
                const uint32_t wend = n + 32u * nch;
                const uint32_t* tw = win + lane;
#pragma unroll 1
                for (; n < wend; n += 32u, tw += 32) {
                    const float dch = drive_at(n + 1u + lane, P);
                    uint32_t pm[PPT] = {0u, 0u}, dm[PPT];
                    float z0[PPT] = {0.0f, 0.0f}, z1[PPT] = {0.0f, 0.0f}, z2[PPT] = {0.0f, 0.0f};
                    dm[0] = tw[0];                           // state at each step of the chunk
                    dm[1] = tw[kWinChunks * 32u];
                    chunk_steps_x2<POIS, DICH, GAUSS, ACC>(S, P, K, path, n, dch, dcur, w, pm, z0, z1, z2,
                                                           dm);
                    if (ACC && ((n + 32u) & 255u) == 0u) {
#pragma unroll
                        for (int p = 0; p < PPT; ++p) {
                            S[p].svd += (double)S[p].sv;
                            S[p].sv2d += (double)S[p].sv2;
                            S[p].sv = 0.0f;
                            S[p].sv2 = 0.0f;
                        }
                    }
                }
            }
        } else if constexpr (WindowedKicks2<MODEL, POIS, DICH, GAUSS, PPT>::value) {
            // chunks in windows of up to kKick2Chunks, kicks drawn at the start of each
            uint32_t* tw0 = win + lane;
            uint32_t* tw1 = win + kKick2WordsPerLane * 32u + lane;
            const float* tq[2] = {(const float*)(tw0 + kKick2Chunks * 32u),
                                  (const float*)(tw1 + kKick2Chunks * 32u)};
            while (n + 32u <= n_end) {
                uint32_t wend = n + 32u * min(kKick2Chunks, (n_end - n) >> 5);
                uint32_t es[2], js[2], w2s[2], w3s[2];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    es[p] = S[p].eP; js[p] = S[p].JP; w2s[p] = S[p].pw2; w3s[p] = S[p].pw3;
                }
                const uint32_t c0 = window_kicks<kKick2Chunks, kKick2Queue>(S[0], P, K, path[0], n, wend, tw0);
                const uint32_t c1 = window_kicks<kKick2Chunks, kKick2Queue>(S[1], P, K, path[1], n, wend, tw1);
                const uint32_t cover = __reduce_min_sync(0xffffffffu, min(c0, c1));
                if (cover < wend) {
                    // some lane's queue filled up: draw again from the saved events
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        S[p].eP = es[p]; S[p].JP = js[p]; S[p].pw2 = w2s[p]; S[p].pw3 = w3s[p];
                    }
                    if (cover < n + 32u) {
                        // more kicks within the next chunk than a queue holds:
                        // that chunk with its events drawn per chunk
                        chunk_drawn_per_chunk<MODEL, POIS, DICH, GAUSS, ACC, PPT>(S, P, K, path, lane, n, dcur, w);
                        n += 32u;
                        continue;
                    }
                    wend = n + ((cover - n) & ~31u);      // the whole chunks every lane covers
                    window_kicks<kKick2Chunks, kKick2Queue>(S[0], P, K, path[0], n, wend, tw0);
                    window_kicks<kKick2Chunks, kKick2Queue>(S[1], P, K, path[1], n, wend, tw1);
                }
                const float* qp[2] = {tq[0], tq[1]};
                float zq[2] = {tq[0][0], tq[1][0]};
#pragma unroll 1
                for (const uint32_t* pmw = tw0; n < wend; n += 32u, pmw += 32) {
                    const float dch = drive_at(n + 1u + lane, P);
                    uint32_t pm[2] = {pmw[0], pmw[kKick2WordsPerLane * 32u]}, pm_unused[2], dm[2];
                    float z0[2], z1[2], z2[2];
                    chunk_events_multi<false, DICH, PPT>(S, P, K, path, n, pm_unused, z0, z1, z2, dm);
                    chunk_steps_x2<POIS, DICH, GAUSS, ACC, true>(S, P, K, path, n, dch, dcur, w, pm, z0, z1, z2,
                                                                 dm, qp, zq);
                    flush_window_sums<ACC, PPT>(S, n);
                }
            }
        } else
        for (; n + 32u <= n_end; n += 32u)
            chunk_drawn_per_chunk<MODEL, POIS, DICH, GAUSS, ACC, PPT>(S, P, K, path, lane, n, dcur, w);
    }
    if (n < n_end) {
#pragma unroll
        for (int p = 0; p < PPT; ++p)
            single_steps<MODEL, POIS, DICH, GAUSS, ACC>(S[p], P, K, path[p], n, n_end);
    }
}

// win: this warp's kWinWordsPerWarp words of shared memory when
// WindowedFlips holds (else unused).
template <int MODEL, bool POIS, int DICH, int GAUSS, int PPT>
__device__ __forceinline__ void simulate_paths(const PointConsts& P, const LaunchConsts& K,
                                               const uint32_t (&path)[PPT], uint32_t lane,
                                               PathResult (&R)[PPT], uint32_t* win = nullptr)
{
    PathState S[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) init_path<MODEL, POIS, DICH>(S[p], P, K, path[p]);
    run_steps_multi<MODEL, POIS, DICH, GAUSS, false, PPT>(S, P, K, path, lane, 0u, P.n_tr, win);
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if (!FoldPerStep<MODEL>::value) fold<MODEL>(S[p]);
        S[p].c_i = S[p].c;
        S[p].kf_i = S[p].kf;
    }
    run_steps_multi<MODEL, POIS, DICH, GAUSS, MODEL == kModelInertial, PPT>(S, P, K, path, lane, P.n_tr,
                                                                            P.n_tr + P.n_avg, win);
#pragma unroll
    for (int p = 0; p < PPT; ++p) finish_path<MODEL, POIS, DICH>(S[p], P, R[p]);
}

// ---------------------------------------------------------------- saved state

// Path states of a segmented run in global memory (Algorithm 5 keeps the
// state in registers within a launch and in global memory between launches):
// structure of arrays, `stride` paths per plane (a multiple of 32, so each
// warp's loads and stores are whole 128-byte lines).  Planes: 2 FP64 (svd,
// sv2d), then 7 FP32 (c, v, kf, c_i, kf_i, sv, sv2), then 10 u32 (eP, JP, pw2,
// pw3, eD, JD, dst, dw1, dw2, dw3): 84 bytes per path.
constexpr uint32_t kStateBytesPerPath = 84u;

struct StatePlanes {
    unsigned char* base;
    uint32_t stride;
    __device__ __forceinline__ double* d(int k) const { return (double*)base + (size_t)k * stride; }
    __device__ __forceinline__ float* f(int k) const
    {
        return (float*)(base + 16ull * stride) + (size_t)k * stride;
    }
    __device__ __forceinline__ uint32_t* u(int k) const
    {
        return (uint32_t*)(base + 44ull * stride) + (size_t)k * stride;
    }
};

__device__ __forceinline__ void load_state(PathState& S, const StatePlanes& M, uint32_t path)
{
    S.svd = M.d(0)[path]; S.sv2d = M.d(1)[path];
    S.c = M.f(0)[path]; S.v = M.f(1)[path]; S.kf = M.f(2)[path];
    S.c_i = M.f(3)[path]; S.kf_i = M.f(4)[path]; S.sv = M.f(5)[path]; S.sv2 = M.f(6)[path];
    S.eP = M.u(0)[path]; S.JP = M.u(1)[path]; S.pw2 = M.u(2)[path]; S.pw3 = M.u(3)[path];
    S.eD = M.u(4)[path]; S.JD = M.u(5)[path]; S.dst = M.u(6)[path];
    S.dw1 = M.u(7)[path]; S.dw2 = M.u(8)[path]; S.dw3 = M.u(9)[path];
}

__device__ __forceinline__ void store_state(const PathState& S, const StatePlanes& M, uint32_t path)
{
    M.d(0)[path] = S.svd; M.d(1)[path] = S.sv2d;
    M.f(0)[path] = S.c; M.f(1)[path] = S.v; M.f(2)[path] = S.kf;
    M.f(3)[path] = S.c_i; M.f(4)[path] = S.kf_i; M.f(5)[path] = S.sv; M.f(6)[path] = S.sv2;
    M.u(0)[path] = S.eP; M.u(1)[path] = S.JP; M.u(2)[path] = S.pw2; M.u(3)[path] = S.pw3;
    M.u(4)[path] = S.eD; M.u(5)[path] = S.JD; M.u(6)[path] = S.dst;
    M.u(7)[path] = S.dw1; M.u(8)[path] = S.dw2; M.u(9)[path] = S.dw3;
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Pull the next warp item, or the first of `count` consecutive items (lane 0
// increments the counter); UINT32_MAX = done.
// With a budget, a warp that has run longer than it since t0 takes no further
// item and marks the launch as timed out (the host reads the status word).
__device__ __forceinline__ uint32_t next_item(uint32_t* counter, int32_t* status,
                                              const LaunchConsts& K, uint32_t lane, uint64_t t0,
                                              uint32_t count = 1u)
{
    uint32_t item = 0u;
    if (lane == 0u) {
        if (K.budget_ns != 0ull && globaltimer_ns() - t0 > K.budget_ns) {
            atomicExch(status, kStatusTimedOut);
            item = 0xffffffffu;
        } else {
            item = atomicAdd(counter, count);
        }
    }
    item = __shfl_sync(0xffffffffu, item, 0);
    return item < K.n_items ? item : 0xffffffffu;
}

// Write one item's FP64 partial sums {paths, sum vbar, sum vbar^2, sum v, sum v^2}.
__device__ __forceinline__ void store_partial(double* partials, uint32_t item, uint32_t lane,
                                              bool valid, const PathResult& R)
{
    const double n = warp_sum(valid ? 1.0 : 0.0);
    const double s1 = warp_sum(valid ? R.vbar : 0.0);
    const double s2 = warp_sum(valid ? __dmul_rn(R.vbar, R.vbar) : 0.0);
    const double s3 = warp_sum(valid ? R.sum_v : 0.0);
    const double s4 = warp_sum(valid ? R.sum_v2 : 0.0);
    if (lane == 0u) {
        double* o = partials + 5ull * item;
        o[0] = n; o[1] = s1; o[2] = s2; o[3] = s3; o[4] = s4;
    }
}

__device__ __forceinline__ void store_path(const PathOutPtrs& po, uint32_t path, const PathResult& R)
{
    if (po.X_f) po.X_f[path] = R.X_f;
    if (po.v_f) po.v_f[path] = R.v_f;
    if (po.vbar) po.vbar[path] = R.vbar;
    if (po.jP) po.jP[path] = R.jP;
    if (po.jD) po.jD[path] = R.jD;
}

}  // namespace sde
