/*
 * sde_oracle.h -- plain FP64 CPU oracle for the Brownian-motor Monte Carlo
 * method of Spiechowicz, Kostur & Machura, "GPU accelerated Monte Carlo
 * simulation of Brownian motors dynamics with CUDA" (arXiv:1409.4923).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the independent checker of the CUDA
 * engine.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs may load or call it.  It shares no code, header, table or
 * constant generator with the CUDA engine; the two only agree on the random
 * stream contract written out below, each implementing it on its own.
 *
 * What it computes: Algorithms 1-4 of Sec. 4 step by step, in double
 * precision, with no blocking, fusion or reordering, for
 *   - the inertial tilted, driven washboard (state x, v):
 *       x' = v,  v' = -g v - V0 2pi cos(2pi x) + a cos(w t) + F + noise,
 *     Gaussian intensity G = sqrt(2 g Q);
 *   - the overdamped washboard  x' = -V0 2pi cos(2pi x) + a cos(w t) + F + noise,
 *     G = sqrt(2 Q)  (D_G = Q);
 *   - the overdamped symmetric piecewise-linear potential of period L = 2
 *     (Sec. 3, Eq. 2) with the same drive terms, G = sqrt(2 Q);
 *   - a linear test force x' = -k x + noise (the Ornstein-Uhlenbeck check of
 *     Algorithm 1; the CUDA engine has no such model).
 * Noise: Gaussian white (Algorithm 2 three-point law, Eq. 25, or Gaussian
 * increments), white Poissonian (Algorithm 3, Eqs. 3-8, 26-27), dichotomous
 * (Algorithm 4, Eqs. 13-17, 29-30); all enter the velocity of the inertial
 * model and the position of the overdamped ones.  The jump increments enter
 * the corrector only (Algorithm 1); with ORC_DICHOT_IN_DRIFT the dichotomous
 * force is instead a drift term, constant over the step.
 *
 * Random stream contract (Philox4x32-10 of Salmon et al., SC'11):
 *   key     = (seed & 0xffffffff, seed >> 32)
 *   counter = (idx & 0xffffffff, (tag << 30) | point, path, idx >> 32)
 *   tags    INIT = 0, GAUSS = 1, POIS = 2, DICH = 3
 *   phi(w)  = (w >> 8) * 2^-24 in [0,1);   u(w) = 1 - phi(w) in (0,1]
 *   INIT  idx 0: x0 = x0_lo + (x0_hi - x0_lo) phi(w0)
 *                v0 = v0_lo + (v0_hi - v0_lo) phi(w1)
 *                d0 = 1 (state F_b) iff phi(w2) < mu_a / (mu_a + mu_b)
 *   GAUSS three-point (Alg. 2): step n uses word (n >> 2) & 3 of idx n >> 4,
 *         r = 6^(n & 3) word mod 2^32; -c if r 2^-32 <= 1/6, +c if <= 1/3,
 *         else 0, c = G sqrt(3 dt)
 *   GAUSS Gaussian: idx n >> 2; words (0,1) serve steps 4i, 4i+1 and words
 *         (2,3) steps 4i+2, 4i+3; R = sqrt(-2 ln u(first)), T = 2 pi
 *         phi(second); even step R cos T, odd step R sin T; increment
 *         G sqrt(dt) N
 *   POIS event j (j = 0 is the initial countdown): idx j >> 1, words
 *         2(j&1) and 2(j&1)+1:  wait_j = floor(-ln u(wa) / (lambda dt)),
 *         z_j = -zeta ln u(wb)
 *   DICH event j (j = 0 is the initial countdown): idx j >> 2, word j & 3:
 *         wait_j = floor(-ln u(w) / (mu_new dt)), mu_new the rate of leaving
 *         the state entered at event j (mu_a for -F_a, mu_b for F_b)
 */
#ifndef SDE_ORACLE_H
#define SDE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_INERTIAL_WASHBOARD = 0, ORC_OVERDAMPED_WASHBOARD = 1,
       ORC_OVERDAMPED_PWL = 2, ORC_OVERDAMPED_LINEAR = 3 };

enum { ORC_GAUSS = 1u, ORC_POISSON = 2u, ORC_DICHOT = 4u,
       ORC_GAUSS_NORMAL = 8u, ORC_POIS_COMPENSATED = 16u,
       ORC_DICHOT_IN_DRIFT = 32u   /* Gamma(t) as a drift term, not a corrector increment */ };

typedef struct {
    double gamma, a, omega, F, Q;
    double lambda, zeta;
    double Fa, Fb, mua, mub;
    double V0;               /* potential amplitude; for the linear force: k */
    double x0_lo, x0_hi, v0_lo, v0_hi;
    uint32_t noise;          /* ORC_* flags */
    uint32_t point;          /* point id in the random counter, < 2^30 */
} orc_params;

typedef struct {
    double X_f;        /* unfolded final position x(t_f)                */
    double v_f;        /* final velocity (inertial) else NaN             */
    double X_i;        /* unfolded position at t_i = n_transient dt     */
    double vbar;       /* (x(t_f) - x(t_i)) / (t_f - t_i), Eq. 31 summand */
    double sum_v;      /* sum of v after each averaged step (inertial)   */
    double sum_v2;     /* sum of v^2 after each averaged step            */
    double kink_min;   /* min distance of a PWL force evaluation to a kink */
    double evt_margin; /* min distance of a waiting-time quotient to an integer */
    uint64_t jP, jD;   /* index of the last Poisson / dichotomous event drawn */
    int32_t d;         /* final dichotomous state (1 = F_b)              */
    int32_t pad;
} orc_path_out;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox_many(const uint32_t* ctr, uint64_t n, const uint32_t key[2], uint32_t* out);

/* Integrate paths path0 .. path0+npaths-1 for n_transient + n_avg steps of dt.
 * nthreads <= 0 uses one thread.  Returns 0, or -1 on invalid arguments. */
int orc_run_paths(int model, const orc_params* p, uint64_t seed, uint64_t path0,
                  uint64_t npaths, double dt, uint64_t n_transient, uint64_t n_avg,
                  int nthreads, orc_path_out* out);

/* Sec. 4's local-error indicator chi = (predictor) - (corrector) of every
 * step, without the jump increments, over n_steps steps of paths path0 ..
 * path0 + npaths - 1 from their initial states: out4 = {sum chi_x^2,
 * sum chi_v^2, max |chi_x|, max |chi_v|} over all paths and steps (x in x
 * units; v components zero for the overdamped models).  Returns 0 or -1. */
int orc_local_error(int model, const orc_params* p, uint64_t seed, uint64_t path0,
                    uint64_t npaths, double dt, uint64_t n_steps, int nthreads, double out4[4]);

/* Ensemble statistics of Eq. 31 over n path records:
 * res = {n, mean vbar, sample variance of vbar, stderr, time mean of v,
 *        time variance of v, sum vbar, sum vbar^2}. */
void orc_stats(const orc_path_out* out, uint64_t n, uint64_t n_avg, double res[8]);

/* Per-step noise increments of one path, n steps (for the noise pins).
 * kind: 1 Gaussian (Alg. 2), 2 Poissonian (Alg. 3, Delta eta_n),
 *       3 dichotomous (Alg. 4, Gamma value of step n, i.e. Delta Gamma_n / dt). */
int orc_noise_sequence(int kind, int model, const orc_params* p, uint64_t seed,
                       uint64_t path, double dt, uint64_t n, double* out);

/* Stream helpers exposed for the tests. */
void orc_stream_words(uint64_t seed, uint32_t tag, uint32_t point, uint32_t path,
                      uint64_t idx, uint32_t out[4]);

#ifdef __cplusplus
}
#endif
#endif
