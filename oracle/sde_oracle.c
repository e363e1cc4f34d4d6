/*
 * sde_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see the
 * header for who may call it and for the random stream contract).
 *
 * Every function follows the paper (Spiechowicz, Kostur & Machura,
 * arXiv:1409.4923) step by step; nothing is blocked, fused or reordered.
 * Pins: tests/test_oracle_*.py check it against closed forms and exact
 * laws (free diffusion, Ornstein-Uhlenbeck recursion, Stratonovich velocity,
 * Eqs. 21-23, Poisson counts, dichotomous correlation, equipartition).
 */
#include "sde_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586476925286766559

/* ---------------------------------------------------------------- Philox */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications with
 * the published multipliers, a Weyl key schedule between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The same generator over n counters ctr[4 i .. 4 i + 3] (for bulk tests). */
void orc_philox_many(const uint32_t* ctr, uint64_t n, const uint32_t key[2], uint32_t* out)
{
    for (uint64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

enum { TAG_INIT = 0, TAG_GAUSS = 1, TAG_POIS = 2, TAG_DICH = 3 };

void orc_stream_words(uint64_t seed, uint32_t tag, uint32_t point, uint32_t path,
                      uint64_t idx, uint32_t out[4])
{
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { (uint32_t)(idx & 0xffffffffu), (tag << 30) | point, path,
                        (uint32_t)(idx >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* phi in [0,1) from the top 24 bits; U(0,1) of Algorithms 2-4. */
static double phi24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------ the models */

typedef struct {
    int model;
    orc_params p;
    uint64_t seed;
    uint32_t path;
    double dt;
    double G;          /* Gaussian intensity factor G of Alg. 2 */
    double aP;         /* bias of the Poisson noise, Eq. 6 (or compensated) */
    double kink_min;   /* PWL force: distance of evaluations to the kinks */
} orc_ctx;

/* -V'(x) for the potential of the model.  Washboard V = V0 sin(2 pi x),
 * period 1.  Piecewise-linear V of Eq. 2, period 2: V' = +1 on [-1,0),
 * -1 on [0,1) (mod 2), scaled by V0.  Linear test force: -k x. */
static double minus_dV(orc_ctx* c, double x)
{
    switch (c->model) {
    case ORC_INERTIAL_WASHBOARD:
    case ORC_OVERDAMPED_WASHBOARD:
        return -c->p.V0 * TWO_PI * cos(TWO_PI * x);
    case ORC_OVERDAMPED_PWL: {
        double y = x - 2.0 * floor((x + 1.0) / 2.0);   /* y in [-1, 1) */
        double dist = fabs(y) < 1.0 - fabs(y) ? fabs(y) : 1.0 - fabs(y);
        if (dist < c->kink_min) c->kink_min = dist;
        return y < 0.0 ? -c->p.V0 : c->p.V0;
    }
    default: /* ORC_OVERDAMPED_LINEAR */
        return -c->p.V0 * x;
    }
}

static double drive(const orc_ctx* c, double t)
{
    return c->p.a * cos(c->p.omega * t) + c->p.F;
}

/* ------------------------------------------------------------ the noises */

typedef struct { const orc_ctx* c; uint32_t w[4]; uint64_t idx_cached; int have; } gauss_gen;

/* Algorithm 2 (three-point law, Eq. 25) or Gaussian increments.
 * Three-point law: steps 4i..4i+3 share word i & 3 of Philox index n >> 4;
 * step 4i+k uses r_k = 6^k r_0 mod 2^32, i.e. the uniform phi_k = r_k 2^-32 is
 * frac(6^k phi_0), and Algorithm 2 compares it with 1/6 and 1/3. */
static double gauss_step(gauss_gen* g, uint64_t n)
{
    const orc_ctx* c = g->c;
    const int normal = (c->p.noise & ORC_GAUSS_NORMAL) != 0;
    uint64_t idx = normal ? (n >> 2) : (n >> 4);
    if (!g->have || g->idx_cached != idx) {
        orc_stream_words(c->seed, TAG_GAUSS, c->p.point, c->path, idx, g->w);
        g->idx_cached = idx;
        g->have = 1;
    }
    if (normal) {
        unsigned pair = (unsigned)(n & 3u) >> 1;
        double R = sqrt(-2.0 * log(1.0 - phi24(g->w[2 * pair])));
        double T = TWO_PI * phi24(g->w[2 * pair + 1]);
        double N = (n & 1u) ? R * sin(T) : R * cos(T);
        return c->G * sqrt(c->dt) * N;
    }
    uint32_t r = g->w[(n >> 2) & 3u];
    for (unsigned k = 0; k < (unsigned)(n & 3u); ++k) r *= 6u;     /* mod 2^32 */
    double phi = (double)r * (1.0 / 4294967296.0);
    double step = c->G * sqrt(3.0 * c->dt);
    if (phi <= 1.0 / 6.0) return -step;
    if (phi <= 1.0 / 3.0) return step;
    return 0.0;
}

static void note_margin(double q, double* margin)
{
    double d = q - floor(q);
    if (1.0 - d < d) d = 1.0 - d;
    if (d < *margin) *margin = d;
}

typedef struct { const orc_ctx* c; int64_t s; uint64_t j; double margin; } pois_gen;

/* Waiting time and amplitude of Poisson event j (the event branch of Alg. 3). */
static void pois_event(pois_gen* g, uint64_t j, int64_t* wait, double* z)
{
    const orc_ctx* c = g->c;
    uint32_t w[4];
    orc_stream_words(c->seed, TAG_POIS, c->p.point, c->path, j >> 1, w);
    unsigned k = (unsigned)(j & 1u) * 2u;
    double q = -(1.0 / c->p.lambda) * log(1.0 - phi24(w[k])) / c->dt;
    note_margin(q, &g->margin);
    *wait = (int64_t)floor(q);
    *z = -c->p.zeta * log(1.0 - phi24(w[k + 1]));
}

static void pois_init(pois_gen* g, const orc_ctx* c)
{
    double z0;
    g->c = c; g->j = 0; g->margin = 1.0;
    pois_event(g, 0, &g->s, &z0);   /* initial countdown; amplitude unused */
}

/* Algorithm 3: the Poissonian increment Delta eta_n. */
static double pois_step(pois_gen* g)
{
    const orc_ctx* c = g->c;
    if (g->s <= 0) {
        double z;
        g->j += 1;
        pois_event(g, g->j, &g->s, &z);
        return z - c->aP * c->dt;
    }
    g->s -= 1;
    return -c->aP * c->dt;
}

typedef struct { const orc_ctx* c; int64_t s; uint64_t j; int d; double margin; } dich_gen;

/* Sojourn of event j in the state it enters (the waiting-time draws of Alg. 4). */
static int64_t dich_wait(dich_gen* g, uint64_t j, int state)
{
    const orc_ctx* c = g->c;
    uint32_t w[4];
    orc_stream_words(c->seed, TAG_DICH, c->p.point, c->path, j >> 2, w);
    double mu = state ? c->p.mub : c->p.mua;
    double q = -(1.0 / mu) * log(1.0 - phi24(w[j & 3u])) / c->dt;
    note_margin(q, &g->margin);
    return (int64_t)floor(q);
}

static void dich_init(dich_gen* g, const orc_ctx* c, uint32_t w_init2)
{
    g->c = c; g->j = 0; g->margin = 1.0;
    /* stationary start: P(F_b) = mu_a / (mu_a + mu_b) (Eqs. 14-16) */
    g->d = phi24(w_init2) < c->p.mua / (c->p.mua + c->p.mub) ? 1 : 0;
    g->s = dich_wait(g, 0, g->d);
}

/* Algorithm 4: the dichotomous increment; returns Gamma_n (= Delta Gamma_n / dt). */
static double dich_step(dich_gen* g)
{
    const orc_ctx* c = g->c;
    if (g->s <= 0) {
        g->d = g->d ? 0 : 1;
        g->j += 1;
        g->s = dich_wait(g, g->j, g->d);
    } else {
        g->s -= 1;
    }
    return g->d ? c->p.Fb : -c->p.Fa;
}

/* ------------------------------------------------------------ one path */

static void ctx_setup(orc_ctx* c, int model, const orc_params* p, uint64_t seed,
                      uint32_t path, double dt)
{
    c->model = model;
    c->p = *p;
    c->seed = seed;
    c->path = path;
    c->dt = dt;
    c->G = model == ORC_INERTIAL_WASHBOARD ? sqrt(2.0 * p->gamma * p->Q) : sqrt(2.0 * p->Q);
    if (p->noise & ORC_POIS_COMPENSATED)
        c->aP = p->zeta * (1.0 - exp(-p->lambda * dt)) / dt;
    else
        c->aP = p->lambda * p->zeta;   /* Eq. 6: a = lambda <z> */
    c->kink_min = 1.0;
}

/* chi (may be NULL) accumulates Sec. 4's local-error indicator chi =
 * (predictor) - (corrector) of each step, without the jump increments (which
 * are exact, not discretisation error): chi[0] += chi_x^2, chi[1] += chi_v^2,
 * chi[2] = max |chi_x|, chi[3] = max |chi_v| (v: inertial model only). */
static void run_one(int model, const orc_params* p, uint64_t seed, uint32_t path,
                    double dt, uint64_t n_tr, uint64_t n_avg, orc_path_out* o, double* chi)
{
    orc_ctx c;
    ctx_setup(&c, model, p, seed, path, dt);
    const unsigned nz = p->noise;
    const int inertial = model == ORC_INERTIAL_WASHBOARD;

    uint32_t w0[4];
    orc_stream_words(seed, TAG_INIT, p->point, path, 0, w0);
    double x = p->x0_lo + (p->x0_hi - p->x0_lo) * phi24(w0[0]);
    double v = p->v0_lo + (p->v0_hi - p->v0_lo) * phi24(w0[1]);

    gauss_gen gg = { &c, {0, 0, 0, 0}, 0, 0 };
    pois_gen pg;
    dich_gen dg;
    if (nz & ORC_POISSON) pois_init(&pg, &c);
    if (nz & ORC_DICHOT) dich_init(&dg, &c, w0[2]);

    double X_i = x, sum_v = 0.0, sum_v2 = 0.0;
    const uint64_t n_total = n_tr + n_avg;
    for (uint64_t n = 0; n < n_total; ++n) {
        const double t0 = (double)n * dt, t1 = (double)(n + 1) * dt;
        double dxi = (nz & ORC_GAUSS) ? gauss_step(&gg, n) : 0.0;
        double deta = (nz & ORC_POISSON) ? pois_step(&pg) : 0.0;
        const double gam = (nz & ORC_DICHOT) ? dich_step(&dg) : 0.0;
        /* Gamma_n enters as the corrector increment Delta Gamma_n = Gamma_n dt
         * (Algorithm 1), or, with ORC_DICHOT_IN_DRIFT, as a force term of
         * Eq. 24, constant over the step, in every drift evaluation */
        const double gdrift = (nz & ORC_DICHOT_IN_DRIFT) ? gam : 0.0;
        const double dgam = (nz & ORC_DICHOT_IN_DRIFT) ? 0.0 : gam * dt;

        if (inertial) {
            /* Algorithm 1 applied to y = (x, v); noise acts on v only and the
             * jump increments enter only the corrector. */
            double F1x = v;
            double F1v = -p->gamma * v + minus_dV(&c, x) + drive(&c, t0) + gdrift;
            double xb = x + F1x * dt;
            double vb = v + F1v * dt + dxi;
            double F2x = vb;
            double F2v = -p->gamma * vb + minus_dV(&c, xb) + drive(&c, t1) + gdrift;
            xb = x + 0.5 * (F1x + F2x) * dt;                      /* predictor */
            vb = v + 0.5 * (F1v + F2v) * dt + dxi;
            const double xp = xb, vp = vb;
            F2x = vb;
            F2v = -p->gamma * vb + minus_dV(&c, xb) + drive(&c, t1) + gdrift;
            x = x + 0.5 * (F1x + F2x) * dt;                       /* corrector */
            v = v + 0.5 * (F1v + F2v) * dt + dxi + deta + dgam;
            if (chi) {
                const double cx = xp - x, cv = vp - (v - deta - dgam);
                chi[0] += cx * cx;
                chi[1] += cv * cv;
                if (fabs(cx) > chi[2]) chi[2] = fabs(cx);
                if (fabs(cv) > chi[3]) chi[3] = fabs(cv);
            }
        } else {
            double F1 = minus_dV(&c, x) + drive(&c, t0) + gdrift;
            double xb = x + F1 * dt + dxi;
            double F2 = minus_dV(&c, xb) + drive(&c, t1) + gdrift;
            xb = x + 0.5 * (F1 + F2) * dt + dxi;                  /* predictor */
            F2 = minus_dV(&c, xb) + drive(&c, t1) + gdrift;
            x = x + 0.5 * (F1 + F2) * dt + dxi + deta + dgam;     /* corrector */
            if (chi) {
                const double cx = xb - (x - deta - dgam);
                chi[0] += cx * cx;
                if (fabs(cx) > chi[2]) chi[2] = fabs(cx);
            }
        }
        if (n + 1 == n_tr) X_i = x;
        if (n + 1 > n_tr && inertial) {
            sum_v += v;
            sum_v2 += v * v;
        }
    }
    o->X_f = x;
    o->v_f = inertial ? v : NAN;
    o->X_i = X_i;
    o->vbar = n_avg ? (x - X_i) / ((double)n_avg * dt) : NAN;
    o->sum_v = sum_v;
    o->sum_v2 = sum_v2;
    o->kink_min = c.kink_min;
    o->evt_margin = 1.0;
    o->jP = 0; o->jD = 0; o->d = 0; o->pad = 0;
    if (nz & ORC_POISSON) { o->jP = pg.j; if (pg.margin < o->evt_margin) o->evt_margin = pg.margin; }
    if (nz & ORC_DICHOT) {
        o->jD = dg.j; o->d = dg.d;
        if (dg.margin < o->evt_margin) o->evt_margin = dg.margin;
    }
}

/* ------------------------------------------------------------ threading */

typedef struct {
    int model; const orc_params* p; uint64_t seed; uint64_t first, count;
    double dt; uint64_t n_tr, n_avg; orc_path_out* out; double* chi;
} orc_job;

static void* orc_worker(void* arg)
{
    orc_job* jb = (orc_job*)arg;
    for (uint64_t i = 0; i < jb->count; ++i)
        run_one(jb->model, jb->p, jb->seed, (uint32_t)(jb->first + i), jb->dt,
                jb->n_tr, jb->n_avg, jb->out + i, jb->chi ? jb->chi + 4 * i : NULL);
    return NULL;
}

static int run_paths_impl(int model, const orc_params* p, uint64_t seed, uint64_t path0,
                          uint64_t npaths, double dt, uint64_t n_tr, uint64_t n_avg,
                          int nthreads, orc_path_out* out, double* chi);

int orc_run_paths(int model, const orc_params* p, uint64_t seed, uint64_t path0,
                  uint64_t npaths, double dt, uint64_t n_tr, uint64_t n_avg,
                  int nthreads, orc_path_out* out)
{
    return run_paths_impl(model, p, seed, path0, npaths, dt, n_tr, n_avg, nthreads, out, NULL);
}

int orc_local_error(int model, const orc_params* p, uint64_t seed, uint64_t path0,
                    uint64_t npaths, double dt, uint64_t n_steps, int nthreads, double out4[4])
{
    if (!out4) return -1;
    out4[0] = out4[1] = out4[2] = out4[3] = 0.0;
    if (npaths == 0) return 0;
    orc_path_out* po = (orc_path_out*)calloc((size_t)npaths, sizeof(orc_path_out));
    double* chi = (double*)calloc((size_t)npaths * 4, sizeof(double));
    if (!po || !chi) { free(po); free(chi); return -1; }
    int rc = run_paths_impl(model, p, seed, path0, npaths, dt, 0, n_steps, nthreads, po, chi);
    if (rc == 0) {
        for (uint64_t i = 0; i < npaths; ++i) {       /* fixed order */
            out4[0] += chi[4 * i];
            out4[1] += chi[4 * i + 1];
            if (chi[4 * i + 2] > out4[2]) out4[2] = chi[4 * i + 2];
            if (chi[4 * i + 3] > out4[3]) out4[3] = chi[4 * i + 3];
        }
    }
    free(po);
    free(chi);
    return rc;
}

static int run_paths_impl(int model, const orc_params* p, uint64_t seed, uint64_t path0,
                          uint64_t npaths, double dt, uint64_t n_tr, uint64_t n_avg,
                          int nthreads, orc_path_out* out, double* chi)
{
    if (!p || !out || !(dt > 0.0) || model < 0 || model > ORC_OVERDAMPED_LINEAR) return -1;
    if (path0 + npaths > 0x100000000ull || p->point >= (1u << 30)) return -1;
    if (npaths == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > npaths) nthreads = (int)npaths;
    orc_job* jobs = (orc_job*)calloc((size_t)nthreads, sizeof(orc_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    uint64_t per = npaths / (uint64_t)nthreads, extra = npaths % (uint64_t)nthreads, at = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t cnt = per + ((uint64_t)t < extra ? 1 : 0);
        orc_job jb = { model, p, seed, path0 + at, cnt, dt, n_tr, n_avg, out + at, chi ? chi + 4 * at : NULL };
        jobs[t] = jb;
        at += cnt;
    }
    int* made = (int*)calloc((size_t)nthreads, sizeof(int));
    for (int t = 1; t < nthreads; ++t)
        made[t] = made ? pthread_create(&th[t], NULL, orc_worker, &jobs[t]) == 0 : 0;
    orc_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) {
        if (made && made[t]) pthread_join(th[t], NULL);
        else orc_worker(&jobs[t]);          /* no thread: run that share inline */
    }
    free(made);
    free(jobs);
    free(th);
    return 0;
}

/* ------------------------------------------------------------ statistics */

/* Eq. 31: <v> as the ensemble mean of the per-path quotients; two-pass
 * sample variance in long double; time averages over all averaged steps. */
void orc_stats(const orc_path_out* out, uint64_t n, uint64_t n_avg, double res[8])
{
    long double s = 0.0L, s2 = 0.0L, tv = 0.0L, tv2 = 0.0L;
    for (uint64_t i = 0; i < n; ++i) {
        s += out[i].vbar;
        s2 += (long double)out[i].vbar * out[i].vbar;
        tv += out[i].sum_v;
        tv2 += out[i].sum_v2;
    }
    long double mean = n ? s / (long double)n : 0.0L;
    long double m2 = 0.0L;
    for (uint64_t i = 0; i < n; ++i) {
        long double d = out[i].vbar - mean;
        m2 += d * d;
    }
    long double var = n > 1 ? m2 / (long double)(n - 1) : 0.0L;
    long double cnt = (long double)n * (long double)n_avg;
    long double tmean = cnt > 0 ? tv / cnt : 0.0L;
    res[0] = (double)n;
    res[1] = (double)mean;
    res[2] = (double)var;
    res[3] = n ? (double)sqrtl(var / (long double)n) : 0.0;
    res[4] = (double)tmean;
    res[5] = cnt > 0 ? (double)(tv2 / cnt - tmean * tmean) : 0.0;
    res[6] = (double)s;
    res[7] = (double)s2;
}

/* ------------------------------------------------------------ noise pins */

int orc_noise_sequence(int kind, int model, const orc_params* p, uint64_t seed,
                       uint64_t path, double dt, uint64_t n, double* out)
{
    if (!p || !out || !(dt > 0.0) || path >= 0x100000000ull) return -1;
    orc_ctx c;
    ctx_setup(&c, model, p, seed, (uint32_t)path, dt);
    uint32_t w0[4];
    orc_stream_words(seed, TAG_INIT, p->point, (uint32_t)path, 0, w0);
    if (kind == 1) {
        gauss_gen gg = { &c, {0, 0, 0, 0}, 0, 0 };
        for (uint64_t i = 0; i < n; ++i) out[i] = gauss_step(&gg, i);
    } else if (kind == 2) {
        pois_gen pg;
        pois_init(&pg, &c);
        for (uint64_t i = 0; i < n; ++i) out[i] = pois_step(&pg);
    } else if (kind == 3) {
        dich_gen dg;
        dich_init(&dg, &c, w0[2]);
        for (uint64_t i = 0; i < n; ++i) out[i] = dich_step(&dg);
    } else {
        return -1;
    }
    return 0;
}
