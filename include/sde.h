/*
 * sde.h -- C ABI of the GB300 (sm_103a) Brownian-motor Monte Carlo engine.
 *
 * The engine integrates many independent realisations of a Langevin equation
 * with the jump-adapted simplified weak-order-2.0 predictor-corrector scheme
 * (Algorithm 1) driven by Gaussian white noise (Algorithm 2, Eq. 25), white
 * Poissonian noise (Algorithm 3, Eqs. 3-8 and 26-27) and dichotomous noise
 * (Algorithm 4, Eqs. 13-17 and 29-30), and reduces them to the ensemble
 * average of Eq. 31 (mean velocity, its variance and standard error) and to
 * time-and-ensemble velocity moments.  Every step of that path runs in the
 * library's own CUDA kernels; there is no CPU fallback.
 *
 * Models (x is the coordinate, V = V0 sin(2 pi x) has period L = 1, the
 * piecewise-linear V of Eq. 2 has period L = 2):
 *   SDE_INERTIAL_WASHBOARD    x' = v,
 *                             v' = -gamma v - V'(x) + a cos(omega t) + F
 *                                  + sqrt(2 gamma Q) xi(t) + eta(t) + Gamma(t)
 *   SDE_OVERDAMPED_WASHBOARD  x' = -V'(x) + a cos(omega t) + F
 *                                  + sqrt(2 Q) xi(t) + eta(t) + Gamma(t)
 *   SDE_OVERDAMPED_PWL        as the previous line with V of Eq. 2 (Eq. 24;
 *                             Models I and II are its limits, Eqs. 1 and 12)
 * Noise is added to v (inertial) or x (overdamped).  The Poissonian and
 * dichotomous increments enter only the corrector (Algorithm 1), unless
 * SDE_DICHOT_IN_DRIFT makes the dichotomous force a drift term.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = the 64-bit seed,
 * counter = (index_lo, tag << 30 | point, path, index_hi); tag 0 initial
 * state, 1 Gaussian (three-point law: word (n >> 2) & 3 of index n >> 4,
 * multiplied by 6^(n & 3) modulo 2^32, serves step n; Gaussian increments:
 * words of index n >> 2), 2 Poisson (event j: words 2(j&1), 2(j&1)+1 of index
 * j >> 1), 3 dichotomous (event j: word j & 3 of index j >> 2).  Uniforms are phi = (w >> 8) 2^-24 in [0,1) and
 * u = 1 - phi in (0,1].  Results are a pure function of (model, parameters,
 * seed, path count, dt, step counts); they do not depend on the launch shape.
 *
 * Errors: every int-returning call returns 0 on success or a negative SDE_E*
 * code; sde_last_error() gives the message.  Nothing throws across the ABI.
 * Threading: one context must not be used from two host threads at once.
 */
#ifndef SDE_H
#define SDE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SDE_OK         0
#define SDE_EINVAL    -1   /* invalid argument (NaN parameter, dt <= 0, ...) */
#define SDE_ECUDA     -2   /* a CUDA call failed (message names it)           */
#define SDE_ENOMEM    -3   /* device or host allocation failed                */
#define SDE_ETIMEDOUT -4   /* the device-side deadline expired before the end */
#define SDE_ESTATE    -5   /* call out of order (e.g. stats before run)        */

typedef enum {
    SDE_INERTIAL_WASHBOARD = 0,
    SDE_OVERDAMPED_WASHBOARD = 1,
    SDE_OVERDAMPED_PWL = 2
} sde_model;

/* noise_flags */
#define SDE_NOISE_GAUSS       1u   /* Gaussian white noise, intensity Q          */
#define SDE_NOISE_POISSON     2u   /* white Poissonian noise (lambda, zeta)      */
#define SDE_NOISE_DICHOT      4u   /* dichotomous noise (-Fa, Fb; mua, mub)      */
#define SDE_GAUSS_NORMAL      8u   /* Gaussian increments instead of Eq. 25      */
#define SDE_POIS_COMPENSATED 16u   /* bias a = zeta (1 - e^{-lambda dt}) / dt    */
                                   /* instead of Eq. 6's lambda zeta             */
#define SDE_DICHOT_IN_DRIFT  32u   /* the dichotomous force Gamma(t) as a drift  */
                                   /* term in all three drift evaluations of     */
                                   /* Algorithm 1 instead of a corrector         */
                                   /* increment; needs SDE_NOISE_DICHOT          */

/* Parameters of one point of parameter space.  Plain old data; the library
 * copies it at the call.  Rates and intensities must be finite and >= 0;
 * lambda > 0 and zeta > 0 with SDE_NOISE_POISSON; Fa, Fb >= 0 and mua,
 * mub > 0 with SDE_NOISE_DICHOT.  The initial state of path i is
 * x0 = x0_lo + (x0_hi - x0_lo) phi, v0 = v0_lo + (v0_hi - v0_lo) phi', and
 * the dichotomous state starts in F_b with probability mua / (mua + mub). */
typedef struct {
    double gamma, a, omega, F, Q;   /* damping, drive amplitude/frequency, bias, D_G */
    double lambda, zeta;            /* Poisson rate and mean amplitude (Eqs. 4-5)   */
    double Fa, Fb, mua, mub;        /* dichotomous levels and rates (Eqs. 13-14)    */
    double V0;                      /* amplitude of the potential                   */
    double x0_lo, x0_hi, v0_lo, v0_hi;
    uint32_t noise_flags;
    uint32_t point;                 /* point id in the random counter, < 2^30       */
} sde_params;

/* Ensemble statistics of one run (Eq. 31 and time averages). */
typedef struct {
    uint64_t n;        /* number of paths                                       */
    double mean_v;     /* <(x(t_f) - x(t_i)) / (t_f - t_i)>  (Eq. 31)           */
    double var_v;      /* sample variance of the per-path quotient              */
    double stderr_v;   /* sqrt(var_v / n)                                       */
    double tmean_v;    /* time-and-ensemble mean of v over the averaging window  */
    double tvar_v;     /* time-and-ensemble variance of v (inertial model only) */
    double sums[5];    /* device FP64 sums: n, sum vbar, sum vbar^2, sum v, sum v^2 */
    int32_t status;    /* SDE_OK or SDE_ETIMEDOUT                               */
    int32_t pad;
} sde_stats_t;

/* Optional per-path outputs, all DEVICE pointers of length `paths` (any may
 * be NULL).  X_f: unfolded final position; v_f: final velocity (inertial);
 * vbar: per-path Eq. 31 quotient; jP, jD: index of the last Poisson /
 * dichotomous event drawn (0 = only the initial countdown). */
typedef struct {
    double* X_f;
    float* v_f;
    double* vbar;
    uint32_t* jP;
    uint32_t* jD;
} sde_path_out;

typedef struct sde_ctx sde_ctx;

/* Create a context for `model` with parameters `p` (copied) and `seed`, bound
 * to the CUDA stream `cuda_stream` (a cudaStream_t, borrowed; NULL = legacy
 * default stream) on the current device.  The context owns its device
 * workspace, which grows on demand and is released by sde_destroy.
 * Parameter meaning: Sec. 3 (Eqs. 1-17) and the model list above. */
int sde_create(sde_ctx** out, sde_model model, const sde_params* p, uint64_t seed,
               void* cuda_stream);

/* Replace the parameters of an existing context (validated, copied);
 * parameter meaning as in sde_create.  A convenience for scans driven from
 * the host: no passage of the paper defines this call. */
int sde_set_params(sde_ctx* ctx, const sde_params* p);

/* Enqueue one Monte Carlo run on the context's stream: `paths` independent
 * realisations, each integrated for n_transient + n_avg steps of dt from the
 * initial law above (Algorithm 5: one path per GPU lane, state in registers),
 * then reduced per Eq. 31 with t_i = n_transient dt and t_f = t_i + n_avg dt.
 * Asynchronous: returns after the launches.  paths in [1, 2^32), dt > 0,
 * n_avg >= 1.  EINVAL on bad arguments, ENOMEM / ECUDA on device failure. */
int sde_run(sde_ctx* ctx, uint64_t paths, double dt, uint64_t n_transient, uint64_t n_avg);

/* As sde_run, additionally writing per-path results to `out` (device memory
 * owned by the caller, each array of length `paths`). */
int sde_run_paths(sde_ctx* ctx, uint64_t paths, double dt, uint64_t n_transient,
                  uint64_t n_avg, const sde_path_out* out);

/* As sde_run_paths (out may be NULL) for the realisations first_path ..
 * first_path + paths - 1 of the same ensemble: path i draws its random numbers
 * with counter path index first_path + i, so disjoint ranges run on several
 * GPUs (or one after another) give exactly the per-path results of one run
 * over their union, and the sum of their five FP64 sums (sde_stats_t.sums) is
 * that run's sums up to the order of FP64 addition.  Eq. 31's ensemble
 * average needs nothing else to be shared between ranges.  Per-path outputs
 * are indexed from 0 within the range.  EINVAL if first_path + paths (rounded
 * up to 32) exceeds 2^32. */
int sde_run_range(sde_ctx* ctx, uint64_t first_path, uint64_t paths, double dt,
                  uint64_t n_transient, uint64_t n_avg, const sde_path_out* out);

/* Wait for the last run on the context's stream and return its statistics
 * (host struct `out`).  ESTATE if no run was enqueued. */
int sde_stats(sde_ctx* ctx, sde_stats_t* out);

/* One point of a batched parameter scan: parameters, step size, path count
 * and step counts (transient, averaged). */
typedef struct {
    sde_params p;
    double dt;
    uint64_t paths;
    uint64_t n_transient;
    uint64_t n_avg;
} sde_scan_point;

/* Batched scan (Sec. 5: many parameter values in one kernel call): all
 * `npts` points (host array, copied) run in one persistent launch over
 * (point, 32-path tile) work items ordered longest first, replayed from a
 * CUDA graph when the shape repeats, or as one launch per point on side
 * streams (sde_set_scan_mode), and are folded per point in a fixed order.
 * For the inertial model without Poisson noise an item is 64 paths of one
 * point (two paths per GPU lane on packed FP32 pairs); each 32-path tile still
 * writes its own partial sums, so a point's result equals its single run.
 * All points share the context's model; each point's noise_flags must equal
 * those of the first point.  Writes npts statistics to the host array `out`
 * (synchronises the stream).  deadline_ms > 0 bounds the device time: work
 * items not started by then are skipped and every point's status becomes
 * SDE_ETIMEDOUT (the call then returns SDE_ETIMEDOUT). */
int sde_scan(sde_ctx* ctx, const sde_scan_point* pts, uint32_t npts, sde_stats_t* out,
             double deadline_ms);

/* The batched scan of sde_scan with its results left on the device, for
 * screens that chain on the GPU without a host round trip (Sec. 5: many
 * parameter values per kernel call).  Enqueues the scan on the context's
 * stream and returns without synchronising: the host array pts is copied at
 * the call.  out5 is a caller-owned DEVICE array of 5 * npts doubles that
 * receives, per point in the order of pts, the FP64 sums of sde_stats_t.sums
 * (paths, sum of Eq. 31's quotient, its sum of squares, sum v, sum v^2 over
 * the averaging window); they equal sde_scan's bit for bit.  No deadline.
 * EINVAL on bad arguments (as sde_scan), ENOMEM / ECUDA on device failure. */
int sde_scan_device(sde_ctx* ctx, const sde_scan_point* pts, uint32_t npts, double* out5);

/* Continue the last sde_scan of this context after it returned
 * SDE_ETIMEDOUT: the work items that it did not start run now, under a fresh
 * deadline_ms (0 = none); the items it finished are kept.  Each item's result
 * depends only on its point and paths, so the final statistics equal those of
 * an uninterrupted scan bit for bit.  Writes the statistics of all npts points
 * of that scan to the host array `out`; synchronises the stream.  Returns
 * SDE_ETIMEDOUT again if the new deadline also expires (call it again: every
 * call finishes at least one item per resident warp); SDE_ESTATE if no scan
 * is pending or another call has used the context's workspace since. */
int sde_scan_resume(sde_ctx* ctx, sde_stats_t* out, double deadline_ms);

/* Segmented runs and checkpoints.  Algorithm 5 advances the paths by
 * `samples` steps per kernel call and keeps their state in global memory
 * between calls (Sec. 5: a kernel run-time limit may forbid one launch for
 * the whole simulation).  These calls do the same with a state the caller can
 * also save to host memory and restore in another context or process.  The
 * random numbers are counter-based, so a path's state is its coordinates,
 * period count, window sums and next-event counters; no generator state is
 * saved. */

/* Start a segmented run of the context's current model, parameters and seed;
 * paths, dt, n_transient, n_avg as sde_run.  Allocates the saved states (84
 * bytes per path, path count rounded up to 32) on the device and enqueues
 * nothing.  The run keeps those parameters and that seed: sde_set_params
 * does not change a run in progress.  Replaces any earlier segmented run. */
int sde_begin(sde_ctx* ctx, uint64_t paths, double dt, uint64_t n_transient, uint64_t n_avg);

/* Enqueue one segment: every path advances by min(n_steps, steps left)
 * steps (n_steps = 0: to the end) from its saved state, which is saved again.
 * The segment that reaches n_transient + n_avg also enqueues the Eq. 31
 * reduction (sde_stats then returns the run's statistics) and writes the
 * per-path results to `out` (device arrays as in sde_run_paths; `out` may be
 * NULL).  When every cut point is a multiple of 32 steps or n_transient, the
 * results are bit-identical to those of sde_run / sde_run_paths; other cut
 * points fold x at other steps, which changes FP32 rounding but not the
 * random events.  Calling it on a complete run enqueues the reduction again.
 * *n_done (host, may be NULL) receives the steps done after this segment.
 * Asynchronous.  SDE_ESTATE without sde_begin or sde_restore. */
int sde_advance(sde_ctx* ctx, uint64_t n_steps, const sde_path_out* out, uint64_t* n_done);

/* Size in bytes of a checkpoint of the current segmented run (host output). */
int sde_checkpoint_size(sde_ctx* ctx, uint64_t* bytes);

/* Write a checkpoint of the segmented run into the host buffer `buf` of
 * `bytes` bytes, after waiting for the context's stream: a 224-byte header
 * (magic "SDECKPT1", format version, model, seed, parameters, dt, paths, step
 * counts, steps done, FNV-1a 64 checksum of the states) followed by the saved
 * states in their device layout (structure of arrays).  SDE_EINVAL if bytes is
 * smaller than sde_checkpoint_size; SDE_ESTATE without a segmented run. */
int sde_checkpoint(sde_ctx* ctx, void* buf, uint64_t bytes);

/* Make the checkpoint in the host buffer `buf` (`bytes` bytes, not kept) the
 * context's segmented run, to be continued by sde_advance with the
 * checkpoint's parameters and seed (the context's own stay in force for
 * sde_run and sde_scan).  The context's model must match.  Before anything
 * reaches the device the header, the checksum and every path's event
 * counters (next event at or after the current step, event index >= 1,
 * dichotomous state 0 or 1) are checked: SDE_EINVAL on any mismatch.
 * Synchronises the stream. */
int sde_restore(sde_ctx* ctx, const void* buf, uint64_t bytes);

/* Local-error indicator of Sec. 4: chi = (predictor) - (corrector) of each
 * step, without the jump increments (exact, not discretisation error), over
 * n_steps steps of `paths` paths from their initial states with the
 * context's parameters and seed.  Writes out4 (host) = {rms chi_x (x units),
 * rms chi_v, max |chi_x|, max |chi_v|} over all paths and steps (the v
 * entries are 0 for the overdamped models).  chi is the local error of the
 * second-order scheme: O(dt^3) without noise, O(dt^2.5) with Gaussian noise,
 * so a step size can be chosen per run from two probes (the paper suggests
 * chi for step-size control; the steps of one run stay uniform, as the
 * event streams require).  Synchronises the stream.  EINVAL as sde_run. */
int sde_local_error(sde_ctx* ctx, uint64_t paths, double dt, uint64_t n_steps, double* out4);

/* Reduce `n` device doubles `vals` to {n, sum, sum of squares} with the same
 * FP64 fold the engine uses (pairwise within a warp, Kahan across items).
 * `out3` is a host array of three doubles.  Synchronises the stream.
 * Test aid: it exposes the reduction step of Eq. 31's ensemble average so
 * that it can be checked on its own; the paper has no such call. */
int sde_reduce_f64(sde_ctx* ctx, const double* vals, uint64_t n, double* out3);

/* Words of the engine's device Philox4x32-10 for counters ctr[4*i..4*i+3]
 * (host array) and key (seed): writes 4*n words to the host array `out`.
 * Runs on the device.  Test aid, exposed so that the stream contract can be
 * checked bit for bit; the paper has no such call (it uses cuRAND). */
int sde_philox_words(sde_ctx* ctx, const uint32_t* ctr, uint64_t n, uint64_t seed,
                     uint32_t* out);

/* Launch shape of the path kernels of this context: threads per block
 * (32..128, multiple of 32) and blocks in the grid (0 = one persistent wave
 * from the occupancy calculator).  Results never depend on the shape; the
 * autotuner of the Python layer picks it.  EINVAL outside those ranges.
 * Tuning aid: the paper fixes no launch shape (Sec. 5 only asks for enough
 * threads per block to keep the GPU busy). */
int sde_set_tuning(sde_ctx* ctx, int block_threads, int grid_blocks);

/* Paths integrated by one GPU lane (1 or 2; default 1).  With 2, each lane
 * advances two paths step by step, interleaved, so that their independent
 * dependency chains hide each other's latencies and the drive values and
 * loop work are shared; each path takes exactly the operations it takes with
 * 1, so results do not change.  Applies to sde_run, sde_run_paths and the
 * per-point launches of sde_scan for the overdamped models.  EINVAL otherwise.
 * Tuning aid with no counterpart in the paper, which runs one path per
 * thread (Algorithm 5). */
int sde_set_paths_per_thread(sde_ctx* ctx, int paths_per_thread);

/* How sde_scan runs the points of the inertial model: 0 (default) chooses
 * one point-kernel launch per point when the points have 2048 paths or more
 * on average (64 such launches side by side fill the GPU) and no deadline is
 * given, and the persistent scan kernel otherwise; 1 always the persistent
 * scan kernel; 2 always one launch per point.  With one launch per point a
 * deadline bounds each launch's device time from that launch's own start.  The launches of mode 2 run side by side on side streams of the
 * context, each with its point's constants as kernel arguments.  Results do
 * not depend on the mode.  The other models always run one launch per point.
 * Tuning aid with no counterpart in the paper.  EINVAL outside 0..2. */
int sde_set_scan_mode(sde_ctx* ctx, int mode);

/* Steps per kernel launch of sde_run / sde_run_paths (Algorithm 5's
 * `samples`): 0 (default) runs the whole simulation in one launch; a
 * multiple of 32 cuts it into launches of that many steps, with the path
 * states kept in device memory between them (84 bytes per path, allocated on
 * first use).  Cut points at multiples of 32 steps leave the results
 * bit-identical.  For hosts whose kernels may not run longer than a watchdog
 * limit.  EINVAL if not a multiple of 32. */
int sde_set_steps_per_launch(sde_ctx* ctx, uint64_t steps);

/* Resident blocks per SM of this context's path kernel at `block_threads`
 * (and the context's paths per thread), and the device's SM count (host
 * outputs).  Tuning aid for the autotuner; the paper has no such call. */
int sde_occupancy(sde_ctx* ctx, int block_threads, int* blocks_per_sm, int* sm_count);

/* Largest path count of sde_run_noalloc. */
#define SDE_NOALLOC_MAX_PATHS 2097152u   /* 2^21 */

/* A Monte Carlo run, as sde_run + the device part of sde_stats, that
 * allocates nothing: no cudaMalloc, cudaFree or allocating library call.  For
 * callers that cannot allocate device memory: code under a memory pool or
 * arena that must own every allocation, real-time loops that may not call
 * cudaMalloc / cudaFree (both can synchronise the whole device), hosts that
 * forbid allocation after start-up.  The paper has no counterpart; it is an
 * integration aid.
 *   model, p, seed, paths, dt, n_transient, n_avg: as sde_create + sde_run
 *     (p is a host struct, copied); paths <= SDE_NOALLOC_MAX_PATHS, else
 *     SDE_EINVAL;
 *   cuda_stream: cudaStream_t to enqueue on (NULL = legacy default stream);
 *     the call returns after enqueueing, without synchronising;
 *   out5: caller-owned DEVICE array of 5 doubles that receives the same FP64
 *     sums as sde_stats_t.sums (paths, sum vbar, sum vbar^2, sum v, sum v^2);
 *   status_out: caller-owned DEVICE int32 (or NULL) that receives SDE_OK.
 * Scratch (the work counter, the status word and 5 doubles per 32 paths,
 * 2.6 MB in all) is one file-scope device array of fixed size.  CUDA loads
 * the library's device code on a device lazily, so the array comes into being
 * on a device at the first call there (the driver then reserves it, once) and
 * stays until the process exits.  That first call on each device also looks
 * the array's device address up (cudaGetSymbolAddress): make it at start-up,
 * before any memory arena takes over the device and before any stream
 * capture; later calls allocate nothing.  All calls share the array and it
 * keeps the last call's contents (each call clears what must start at zero),
 * so calls whose work overlaps on the GPU (other streams, other host threads
 * on the same device) race: serialise them.  Errors: SDE_EINVAL, SDE_ECUDA;
 * the message is sde_last_error(NULL) in the calling thread. */
int sde_run_noalloc(sde_model model, const sde_params* p, uint64_t seed, uint64_t paths,
                    double dt, uint64_t n_transient, uint64_t n_avg, void* cuda_stream,
                    double* out5, int32_t* status_out);

/* Free everything the context owns (waits for its stream first). */
void sde_destroy(sde_ctx* ctx);

/* Message of the last error on `ctx`, or, when ctx is NULL, of the last
 * failed call without a context (sde_create, sde_run_noalloc) made by the
 * calling host thread (each thread has its own).  Valid until the next call on
 * the same context (or, for NULL, the next such call in the thread). */
const char* sde_last_error(const sde_ctx* ctx);

/* Library version string (no counterpart in the paper). */
const char* sde_version(void);

#ifdef __cplusplus
}
#endif
#endif
