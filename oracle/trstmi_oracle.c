/*
 * TRSTMI CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision restatement of the stochastic trust-region
 * coherence search (Park, Saltijeral, Zhong, "Grassmannian packings:
 * Trust-region stochastic tuning for matrix incoherence", arXiv 2207.06374).
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library.  It shares no code, header, table
 * or constant generator with the CUDA path; its Philox generator and
 * Box-Muller transform are written here from their published definitions.
 *
 * What is computed (notation of the paper, Sec. "Introduction"):
 *   Phi in C^{d x N} with unit-norm columns phi_j, stored column-major with
 *   interleaved (re, im): phi[2*(j*d + i) + 0] = Re Phi_ij, [.. + 1] = Im.
 *   G = Phi^* Phi,  G_jk = sum_i conj(Phi_ij) Phi_ik  (Gram matrix, Sec. 1).
 *   mu(Phi) = max_{j != k} |G_jk|  (coherence, Sec. 1); by the symmetry
 *   |G_jk| = |G_kj| only j < k is visited (Sec. "Optimization procedure":
 *   the upper-triangular part suffices).  Everything is reduced in |G|^2 and
 *   one square root is taken at the end.
 *   Welch bound mu >= sqrt((N-d)/(d(N-1))) (Sec. "Welch bound ...").
 *
 * The search (Algorithm "TRSTMI optimization steps", step 1 = random unit
 * vectors; the Monte-Carlo sampling of Sec. "Optimization procedure") is read
 * as a derivative-free trust-region iteration.  The paper prints no
 * candidate step or radius rule; the reading used here is:
 *   init:    Phi = normalise_cols(Z_init),  Z_init ~ CN(0,1) entrywise
 *   iter t:  for c < K:  Phi_c = normalise_cols(Phi + Delta * Z_{t,c})
 *            c* = argmin_c mu^2(Phi_c)   (lowest c on ties)
 *            accept iff mu^2(Phi_c*) < mu^2(Phi)   (strict)
 *            accept: Phi <- Phi_c*, Delta <- min(gamma_inc*Delta, Delta_max)
 *            reject: Delta <- max(gamma_dec*Delta, Delta_min)
 *            stop when mu(Phi) <= target or after T iterations.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), key = (seed lo32, seed hi32),
 * counter = (e, c, t, tag) with e = j*ceil(d/2) + (i/2) the index of the pair
 * of entries (i even, i+1) of column j; tag 0 = perturbation, 1 = init (c=t=0).
 * One call gives u0..u3; U = (u + 1/2) 2^-32 in (0,1).  Entry i even uses
 * (u0,u1), i odd uses (u2,u3): Z = sqrt(-ln U_a) * exp(2 pi i U_b), which is
 * the Box-Muller pair (z, z') / sqrt(2), i.e. complex normal CN(0,1).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 round constants as published (SC'11, Sec. 4.2 and Table 2). */
static const uint32_t PHX_M0 = 0xD2511F53u, PHX_M1 = 0xCD9E8D57u;
static const uint32_t PHX_W0 = 0x9E3779B9u, PHX_W1 = 0xBB67AE85u;

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHX_W0; k1 += PHX_W1; }
        uint64_t p0 = (uint64_t)PHX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------- Gaussian entries */

static double u32_to_open01(uint32_t u)
{
    return ((double)u + 0.5) * (1.0 / 4294967296.0);
}

/* Z_ij for the counter slot (c, t, tag); see the header comment. */
void oracle_gauss_entry(uint64_t seed, int d, int i, int j, uint32_t c,
                        uint32_t t, uint32_t tag, double *re, double *im)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t pairs_per_col = (uint32_t)((d + 1) / 2);
    uint32_t ctr[4] = {(uint32_t)j * pairs_per_col + (uint32_t)(i / 2), c, t, tag};
    uint32_t u[4];
    oracle_philox4x32_10(ctr, key, u);
    double ua = (i % 2 == 0) ? u32_to_open01(u[0]) : u32_to_open01(u[2]);
    double ub = (i % 2 == 0) ? u32_to_open01(u[1]) : u32_to_open01(u[3]);
    double r = sqrt(-log(ua));
    double theta = 2.0 * M_PI * ub;
    *re = r * cos(theta);
    *im = r * sin(theta);
}

/* ------------------------------------------------------ columns and Gram */

/* Divide every column by its 2-norm; a zero column is an error (the Remark
 * on normalisation excludes zero columns). */
static int normalise_columns(int N, int d, double *phi)
{
    for (int j = 0; j < N; ++j) {
        double s = 0.0;
        for (int i = 0; i < d; ++i) {
            double a = phi[2 * (j * d + i)], b = phi[2 * (j * d + i) + 1];
            s += a * a + b * b;
        }
        if (!(s > 0.0)) return ORACLE_EINVAL;
        double nrm = sqrt(s);
        for (int i = 0; i < d; ++i) {
            phi[2 * (j * d + i)] /= nrm;
            phi[2 * (j * d + i) + 1] /= nrm;
        }
    }
    return ORACLE_OK;
}

/* |G_jk|^2 with G_jk = sum_i conj(Phi_ij) Phi_ik. */
double oracle_gram_abs2(int d, const double *phi, int j, int k)
{
    double re = 0.0, im = 0.0;
    for (int i = 0; i < d; ++i) {
        double a = phi[2 * (j * d + i)], b = phi[2 * (j * d + i) + 1];
        double x = phi[2 * (k * d + i)], y = phi[2 * (k * d + i) + 1];
        /* (a - ib)(x + iy) = (ax + by) + i(ay - bx) */
        re += a * x + b * y;
        im += a * y - b * x;
    }
    return re * re + im * im;
}

/* mu(Phi)^2 = max_{j<k} |G_jk|^2 by enumerating every pair; 0 if N < 2. */
double oracle_mu2(int N, int d, const double *phi)
{
    double m = 0.0;
    for (int j = 0; j < N; ++j)
        for (int k = j + 1; k < N; ++k) {
            double g = oracle_gram_abs2(d, phi, j, k);
            if (g > m) m = g;
        }
    return m;
}

/* Welch bound sqrt((N-d)/(d(N-1))), clamped at 0 for N <= d. */
double oracle_welch(int N, int d)
{
    if (N <= d || N < 2) return 0.0;
    return sqrt((double)(N - d) / ((double)d * (double)(N - 1)));
}

/* ------------------------------------------------ init and one candidate */

int oracle_init(int N, int d, uint64_t seed, double *phi)
{
    if (N < 1 || d < 1 || !phi) return ORACLE_EINVAL;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < d; ++i)
            oracle_gauss_entry(seed, d, i, j, 0, 0, 1, &phi[2 * (j * d + i)],
                               &phi[2 * (j * d + i) + 1]);
    return normalise_columns(N, d, phi);
}

/* Phi_c = normalise_cols(Phi + delta * Z_{t,c}). */
int oracle_candidate(int N, int d, uint64_t seed, const double *phi,
                     double delta, uint32_t t, uint32_t c, double *out)
{
    if (N < 1 || d < 1 || !phi || !out) return ORACLE_EINVAL;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < d; ++i) {
            double zr, zi;
            oracle_gauss_entry(seed, d, i, j, c, t, 0, &zr, &zi);
            out[2 * (j * d + i)] = phi[2 * (j * d + i)] + delta * zr;
            out[2 * (j * d + i) + 1] = phi[2 * (j * d + i) + 1] + delta * zi;
        }
    return normalise_columns(N, d, out);
}

/* ------------------------------------------- scoring many candidates */

typedef struct {
    int N, d;
    uint64_t seed;
    const double *phi;
    double delta;
    uint32_t t, c0;
    int begin, end;
    double *mu2;
    int status;
} score_job;

static void *score_worker(void *arg)
{
    score_job *jb = (score_job *)arg;
    double *buf = (double *)malloc(sizeof(double) * 2 * (size_t)jb->d * (size_t)jb->N);
    jb->status = ORACLE_OK;
    if (!buf) { jb->status = ORACLE_EINVAL; return NULL; }
    for (int k = jb->begin; k < jb->end; ++k) {
        int st = oracle_candidate(jb->N, jb->d, jb->seed, jb->phi, jb->delta,
                                  jb->t, jb->c0 + (uint32_t)k, buf);
        if (st != ORACLE_OK) { jb->status = st; break; }
        jb->mu2[k] = oracle_mu2(jb->N, jb->d, buf);
    }
    free(buf);
    return NULL;
}

/* mu^2 of candidates c0 .. c0+K-1 of iteration t, split over nthreads. */
int oracle_score(int N, int d, uint64_t seed, const double *phi, double delta,
                 uint32_t t, uint32_t c0, int K, double *mu2, int nthreads)
{
    if (N < 1 || d < 1 || K < 0 || !phi || (K > 0 && !mu2)) return ORACLE_EINVAL;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > K) nthreads = K > 0 ? K : 1;
    score_job *jobs = (score_job *)calloc((size_t)nthreads, sizeof(score_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return ORACLE_EINVAL; }
    for (int w = 0; w < nthreads; ++w) {
        jobs[w] = (score_job){N, d, seed, phi, delta, t, c0,
                              (int)((long long)K * w / nthreads),
                              (int)((long long)K * (w + 1) / nthreads), mu2, 0};
    }
    for (int w = 1; w < nthreads; ++w) pthread_create(&th[w], NULL, score_worker, &jobs[w]);
    score_worker(&jobs[0]);
    for (int w = 1; w < nthreads; ++w) pthread_join(th[w], NULL);
    int st = ORACLE_OK;
    for (int w = 0; w < nthreads; ++w) if (jobs[w].status != ORACLE_OK) st = jobs[w].status;
    free(jobs); free(th);
    return st;
}

/* ---------------------------------- binary32 plain-loop variant (timing)
 * The same scoring in single precision with plain float loops: the frame
 * rounded to float, each candidate entry phi + delta * Z with Z drawn by the
 * same Philox words (U = (u + 1/2) 2^-32 rounded to float, Box-Muller with
 * logf / sqrtf / cosf / sinf), columns normalised in float, mu^2 = max over
 * j < k of |G_jk|^2 accumulated in float.  It serves as the CPU baseline of
 * the binary32 path; its values agree with the binary64 oracle to binary32
 * rounding (the tests pin that), not bit for bit with any GPU kernel. */

static void gauss_entry_f32(uint64_t seed, int d, int i, int j, uint32_t c, uint32_t t,
                            float *re, float *im)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)j * (uint32_t)((d + 1) / 2) + (uint32_t)(i / 2), c, t, 0u};
    uint32_t u[4];
    oracle_philox4x32_10(ctr, key, u);
    float ua = (float)u32_to_open01((i % 2 == 0) ? u[0] : u[2]);
    float ub = (float)u32_to_open01((i % 2 == 0) ? u[1] : u[3]);
    float r = sqrtf(-logf(ua));
    float theta = 6.2831853071795864769f * ub;
    *re = r * cosf(theta);
    *im = r * sinf(theta);
}

typedef struct {
    int N, d;
    uint64_t seed;
    const float *phi;
    float delta;
    uint32_t t, c0;
    int begin, end;
    double *mu2;
    int status;
} score32_job;

static void *score32_worker(void *arg)
{
    score32_job *jb = (score32_job *)arg;
    const int N = jb->N, d = jb->d;
    float *x = (float *)malloc(sizeof(float) * 2 * (size_t)d * (size_t)N);
    jb->status = ORACLE_OK;
    if (!x) { jb->status = ORACLE_EINVAL; return NULL; }
    for (int k = jb->begin; k < jb->end; ++k) {
        const uint32_t c = jb->c0 + (uint32_t)k;
        for (int j = 0; j < N; ++j) {
            float s = 0.0f;
            for (int i = 0; i < d; ++i) {
                float zr, zi;
                gauss_entry_f32(jb->seed, d, i, j, c, jb->t, &zr, &zi);
                float a = jb->phi[2 * (j * d + i)] + jb->delta * zr;
                float b = jb->phi[2 * (j * d + i) + 1] + jb->delta * zi;
                x[2 * (j * d + i)] = a;
                x[2 * (j * d + i) + 1] = b;
                s += a * a + b * b;
            }
            if (!(s > 0.0f)) { jb->status = ORACLE_EINVAL; break; }
            float nrm = sqrtf(s);
            for (int i = 0; i < 2 * d; ++i) x[2 * j * d + i] /= nrm;
        }
        if (jb->status != ORACLE_OK) break;
        float m = 0.0f;
        for (int j = 0; j < N; ++j)
            for (int l = j + 1; l < N; ++l) {
                float gr = 0.0f, gi = 0.0f;
                for (int i = 0; i < d; ++i) {
                    float a = x[2 * (j * d + i)], b = x[2 * (j * d + i) + 1];
                    float e = x[2 * (l * d + i)], f = x[2 * (l * d + i) + 1];
                    gr += a * e + b * f;
                    gi += a * f - b * e;
                }
                float g = gr * gr + gi * gi;
                if (g > m) m = g;
            }
        jb->mu2[k] = (double)m;
    }
    free(x);
    return NULL;
}

/* mu^2 of candidates c0 .. c0+K-1 of iteration t in binary32, split over
 * nthreads (the frame phi is binary64 and rounded to float first). */
int oracle_score_f32(int N, int d, uint64_t seed, const double *phi, double delta,
                     uint32_t t, uint32_t c0, int K, double *mu2, int nthreads)
{
    if (N < 1 || d < 1 || K < 0 || !phi || (K > 0 && !mu2)) return ORACLE_EINVAL;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > K) nthreads = K > 0 ? K : 1;
    float *f = (float *)malloc(sizeof(float) * 2 * (size_t)d * (size_t)N);
    score32_job *jobs = (score32_job *)calloc((size_t)nthreads, sizeof(score32_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!f || !jobs || !th) { free(f); free(jobs); free(th); return ORACLE_EINVAL; }
    for (size_t e = 0; e < 2 * (size_t)d * (size_t)N; ++e) f[e] = (float)phi[e];
    for (int w = 0; w < nthreads; ++w)
        jobs[w] = (score32_job){N, d, seed, f, (float)delta, t, c0,
                                (int)((long long)K * w / nthreads),
                                (int)((long long)K * (w + 1) / nthreads), mu2, 0};
    for (int w = 1; w < nthreads; ++w) pthread_create(&th[w], NULL, score32_worker, &jobs[w]);
    score32_worker(&jobs[0]);
    for (int w = 1; w < nthreads; ++w) pthread_join(th[w], NULL);
    int st = ORACLE_OK;
    for (int w = 0; w < nthreads; ++w) if (jobs[w].status != ORACLE_OK) st = jobs[w].status;
    free(f); free(jobs); free(th);
    return st;
}

/* -------------------------------------------------------- the search */

typedef struct {
    int K;             /* candidates per iteration */
    int T;             /* iteration budget */
    double delta0;     /* initial trust radius */
    double gamma_inc;  /* expansion factor on accept */
    double gamma_dec;  /* contraction factor on reject */
    double delta_min, delta_max;
    double target_mu;  /* stop once mu <= target (<= 0: never) */
} oracle_opts;

typedef struct {
    uint32_t t;        /* iteration counter used for the candidates */
    uint32_t cstar;    /* best candidate */
    double mu2_best;   /* its mu^2 */
    double mu2_cur;    /* mu^2 of Phi after the decision */
    double delta_used; /* radius the candidates were drawn with */
    double delta_next; /* radius after the update */
    int32_t accepted;
    int32_t pad;
} oracle_trace_row;

static void apply_rule(const oracle_opts *o, int accept, double *delta)
{
    if (accept) {
        double v = o->gamma_inc * *delta;
        *delta = v < o->delta_max ? v : o->delta_max;
    } else {
        double v = o->gamma_dec * *delta;
        *delta = v > o->delta_min ? v : o->delta_min;
    }
}

/*
 * Runs iterations t = t0+1 .. t0+T from the state (phi, delta, mu2) in place.
 * Returns the number of iterations done through *iters.  trace may be NULL,
 * else it has room for T rows.
 */
int oracle_search(int N, int d, uint64_t seed, const oracle_opts *o,
                  double *phi, double *delta, double *mu2_cur, uint32_t t0,
                  int *iters, oracle_trace_row *trace, int nthreads)
{
    if (!o || !phi || !delta || !mu2_cur || !iters || o->K < 1 || o->T < 0)
        return ORACLE_EINVAL;
    size_t n = 2 * (size_t)d * (size_t)N;
    double *mu2 = (double *)malloc(sizeof(double) * (size_t)o->K);
    double *cand = (double *)malloc(sizeof(double) * n);
    if (!mu2 || !cand) { free(mu2); free(cand); return ORACLE_EINVAL; }
    double target2 = o->target_mu > 0 ? o->target_mu * o->target_mu : -1.0;
    int done = 0, st = ORACLE_OK;
    for (int it = 0; it < o->T; ++it) {
        if (*mu2_cur <= target2) break;
        uint32_t t = t0 + (uint32_t)it + 1u;
        st = oracle_score(N, d, seed, phi, *delta, t, 0, o->K, mu2, nthreads);
        if (st != ORACLE_OK) break;
        int cstar = 0;
        for (int c = 1; c < o->K; ++c) if (mu2[c] < mu2[cstar]) cstar = c;
        int accept = mu2[cstar] < *mu2_cur;
        double dused = *delta;
        if (accept) {
            st = oracle_candidate(N, d, seed, phi, dused, t, (uint32_t)cstar, cand);
            if (st != ORACLE_OK) break;
            memcpy(phi, cand, sizeof(double) * n);
            *mu2_cur = mu2[cstar];
        }
        apply_rule(o, accept, delta);
        if (trace) {
            trace[it].t = t; trace[it].cstar = (uint32_t)cstar;
            trace[it].mu2_best = mu2[cstar]; trace[it].mu2_cur = *mu2_cur;
            trace[it].delta_used = dused; trace[it].delta_next = *delta;
            trace[it].accepted = accept; trace[it].pad = 0;
        }
        ++done;
    }
    *iters = done;
    free(mu2); free(cand);
    return st;
}

/* Whole run from the seeded initialisation. */
int oracle_run(int N, int d, uint64_t seed, const oracle_opts *o, double *phi,
               double *mu2_out, double *delta_out, int *iters,
               oracle_trace_row *trace, int nthreads)
{
    if (!o || !phi || !mu2_out || !delta_out || !iters) return ORACLE_EINVAL;
    int st = oracle_init(N, d, seed, phi);
    if (st != ORACLE_OK) return st;
    *mu2_out = oracle_mu2(N, d, phi);
    *delta_out = o->delta0;
    return oracle_search(N, d, seed, o, phi, delta_out, mu2_out, 0, iters, trace,
                         nthreads);
}

/*
 * Replays a given sequence of chosen candidates (one per iteration t0+1 ..
 * t0+T): each is regenerated in double precision, scored exactly and put
 * through the accept/radius rule.  Used to check a run whose candidate
 * selection was made elsewhere (e.g. by a reduced-precision screen).
 */
int oracle_replay(int N, int d, uint64_t seed, const oracle_opts *o,
                  double *phi, double *delta, double *mu2_cur, uint32_t t0,
                  int T, const uint32_t *cstar_seq, oracle_trace_row *trace)
{
    if (!o || !phi || !delta || !mu2_cur || T < 0 || (T > 0 && !cstar_seq))
        return ORACLE_EINVAL;
    size_t n = 2 * (size_t)d * (size_t)N;
    double *cand = (double *)malloc(sizeof(double) * n);
    if (!cand) return ORACLE_EINVAL;
    int st = ORACLE_OK;
    for (int it = 0; it < T; ++it) {
        uint32_t t = t0 + (uint32_t)it + 1u;
        double dused = *delta;
        st = oracle_candidate(N, d, seed, phi, dused, t, cstar_seq[it], cand);
        if (st != ORACLE_OK) break;
        double m2 = oracle_mu2(N, d, cand);
        int accept = m2 < *mu2_cur;
        if (accept) { memcpy(phi, cand, sizeof(double) * n); *mu2_cur = m2; }
        apply_rule(o, accept, delta);
        if (trace) {
            trace[it].t = t; trace[it].cstar = cstar_seq[it];
            trace[it].mu2_best = m2; trace[it].mu2_cur = *mu2_cur;
            trace[it].delta_used = dused; trace[it].delta_next = *delta;
            trace[it].accepted = accept; trace[it].pad = 0;
        }
    }
    free(cand);
    return st;
}

/* ------------------------------------------- smooth maximum (log-sum-exp) */

/*
 * The paper's objective (Sec. "Optimization procedure"): the smooth maximum
 *   F_{s,delta}(x) = s + delta * log sum_{i=1}^{n} exp((x_i - s) / delta),
 *   s = max_i x_i,  delta > 0,
 * taken over x = the values |G_jk|^2, j < k, of the frame obtained by
 * dividing each column of the variable V (d x N, complex) by its norm, so
 * n = N(N-1)/2 (Remark on n; Remark on the unconstrained variable).  The
 * Proposition bounds it: s <= F <= s + delta log n.
 *
 * Gradient.  The shift by s cancels (F = delta log sum exp(x_i / delta)
 * identically), so dF/dx_i = w_i = exp((x_i - s)/delta) / sum_l exp((x_l -
 * s)/delta), the softmax weights; the subgradient of the max named in the
 * Remark on the shift contributes (1 - sum_i w_i) = 0 at the argmax.  With
 * phi_k = v_k / r_k (r_k = |v_k|) and G the Hermitian Gram matrix of Phi,
 *   x_jk = G_jk conj(G_jk),  d x_jk / d conj(phi_k) = G_jk phi_j,
 *   d x_jk / d conj(phi_j) = conj(G_jk) phi_k,
 * so the real gradient in Phi, written as a complex array (dF/dRe + i
 * dF/dIm = 2 dF/d conj), is
 *   g_k = 2 sum_{j != k} w_jk G_jk phi_j          (w symmetric, G Hermitian)
 * and through the normalisation (d phi = (dv - phi Re(phi^* dv)) / r)
 *   grad_k = (g_k - phi_k Re(phi_k^* g_k)) / r_k.
 * Frames use the layout of the rest of this file.  grad (2dN doubles) may be
 * NULL.  Returns ORACLE_EINVAL for N < 2, d < 1, delta <= 0 or a zero column.
 */
int oracle_lse(int N, int d, const double *v, double delta, double *F, double *s_out,
               double *grad)
{
    if (N < 2 || d < 1 || !v || !F || !(delta > 0.0)) return ORACLE_EINVAL;
    size_t m = 2 * (size_t)d * (size_t)N;
    size_t n = (size_t)N * (size_t)(N - 1) / 2;
    double *phi = (double *)malloc(sizeof(double) * m);
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double *x = (double *)malloc(sizeof(double) * n);
    int st = ORACLE_OK;
    if (!phi || !r || !x) { st = ORACLE_EINVAL; goto out; }
    memcpy(phi, v, sizeof(double) * m);
    for (int j = 0; j < N; ++j) {
        double q = 0.0;
        for (int i = 0; i < d; ++i) {
            double a = v[2 * (j * d + i)], b = v[2 * (j * d + i) + 1];
            q += a * a + b * b;
        }
        r[j] = sqrt(q);
    }
    st = normalise_columns(N, d, phi);
    if (st != ORACLE_OK) goto out;

    /* x over the pairs j < k in row order, its max s and the shifted sum */
    size_t p = 0;
    double s = 0.0;
    for (int j = 0; j < N; ++j)
        for (int k = j + 1; k < N; ++k, ++p) {
            x[p] = oracle_gram_abs2(d, phi, j, k);
            if (p == 0 || x[p] > s) s = x[p];
        }
    double S = 0.0;
    for (p = 0; p < n; ++p) S += exp((x[p] - s) / delta);
    *F = s + delta * log(S);
    if (s_out) *s_out = s;

    if (grad) {
        double *g = grad;
        memset(g, 0, sizeof(double) * m);
        p = 0;
        for (int j = 0; j < N; ++j)
            for (int k = j + 1; k < N; ++k, ++p) {
                double w = exp((x[p] - s) / delta) / S;
                double gr = 0.0, gi = 0.0;   /* G_jk = sum_i conj(phi_ij) phi_ik */
                for (int i = 0; i < d; ++i) {
                    double a = phi[2 * (j * d + i)], b = phi[2 * (j * d + i) + 1];
                    double c = phi[2 * (k * d + i)], e = phi[2 * (k * d + i) + 1];
                    gr += a * c + b * e;
                    gi += a * e - b * c;
                }
                for (int i = 0; i < d; ++i) {
                    double a = phi[2 * (j * d + i)], b = phi[2 * (j * d + i) + 1];
                    double c = phi[2 * (k * d + i)], e = phi[2 * (k * d + i) + 1];
                    /* g_k += 2 w G_jk phi_j;  g_j += 2 w conj(G_jk) phi_k */
                    g[2 * (k * d + i)] += 2.0 * w * (gr * a - gi * b);
                    g[2 * (k * d + i) + 1] += 2.0 * w * (gr * b + gi * a);
                    g[2 * (j * d + i)] += 2.0 * w * (gr * c + gi * e);
                    g[2 * (j * d + i) + 1] += 2.0 * w * (gr * e - gi * c);
                }
            }
        for (int k = 0; k < N; ++k) {
            double rad = 0.0;   /* Re(phi_k^* g_k) */
            for (int i = 0; i < d; ++i)
                rad += phi[2 * (k * d + i)] * g[2 * (k * d + i)] +
                       phi[2 * (k * d + i) + 1] * g[2 * (k * d + i) + 1];
            for (int i = 0; i < d; ++i) {
                g[2 * (k * d + i)] = (g[2 * (k * d + i)] - phi[2 * (k * d + i)] * rad) / r[k];
                g[2 * (k * d + i) + 1] =
                    (g[2 * (k * d + i) + 1] - phi[2 * (k * d + i) + 1] * rad) / r[k];
            }
        }
    }
out:
    free(phi);
    free(r);
    free(x);
    return st;
}

/* ------------------------------------------------ bounds and diagnostics */

/* Orthoplex bound (Sec. "Conjectures from Numerics", Proposition on the
 * orthoplex and Levenshtein bounds): mu >= 1/sqrt(d) when N > d^2 (d > 1);
 * 0 where it does not apply. */
double oracle_orthoplex(int N, int d)
{
    if (d < 2 || (long long)N <= (long long)d * d) return 0.0;
    return 1.0 / sqrt((double)d);
}

/* Levenshtein bound (same Proposition): mu >= sqrt((2N - d(d+1)) /
 * ((N - d)(d+1))) when N > d^2 (d > 1); 0 where it does not apply. */
double oracle_levenshtein(int N, int d)
{
    if (d < 2 || (long long)N <= (long long)d * d) return 0.0;
    double n = (double)N, dd = (double)d;
    return sqrt((2.0 * n - dd * (dd + 1.0)) / ((n - dd) * (dd + 1.0)));
}

/* max and min of |G_jk|^2 over j < k (N >= 2) by enumerating every pair. */
void oracle_gram_extremes(int N, int d, const double *phi, double *mx, double *mn)
{
    double hi = 0.0, lo = 0.0;
    int first = 1;
    for (int j = 0; j < N; ++j)
        for (int k = j + 1; k < N; ++k) {
            double g = oracle_gram_abs2(d, phi, j, k);
            if (first || g > hi) hi = g;
            if (first || g < lo) lo = g;
            first = 0;
        }
    *mx = hi;
    *mn = lo;
}

/* Number of distinct distances among the |G_jk|, j < k, at resolution tol:
 * each value v falls in bin floor(v / tol), and one distance is a maximal
 * run of consecutive occupied bins.  (The single-distance observation of
 * Sec. "Conjectures from Numerics" counts how many different |<phi_j,
 * phi_k>| a configuration has.)  Returns -1 on bad arguments. */
int oracle_distinct_distances(int N, int d, const double *phi, double tol)
{
    if (N < 2 || d < 1 || !phi || !(tol > 0.0) || tol > 1.0) return -1;
    long nbins = (long)floor(1.0 / tol) + 2;
    unsigned char *occ = (unsigned char *)calloc((size_t)nbins, 1);
    if (!occ) return -1;
    for (int j = 0; j < N; ++j)
        for (int k = j + 1; k < N; ++k) {
            double v = sqrt(oracle_gram_abs2(d, phi, j, k));
            long b = (long)floor(v / tol);
            if (b >= nbins) b = nbins - 1;
            occ[b] = 1;
        }
    int runs = 0;
    for (long b = 0; b < nbins; ++b)
        if (occ[b] && (b == 0 || !occ[b - 1])) ++runs;
    free(occ);
    return runs;
}

/* ------------------------------------- trust-region CG-Steihaug (Alg. 1) */

static double vdot(int n, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* tau >= 0 with |z + tau d| = radius (the root of the quadratic in tau). */
static double to_boundary(int n, const double *z, const double *d, double radius, int pos)
{
    double dd = vdot(n, d, d), zd = vdot(n, z, d), zz = vdot(n, z, z);
    double disc = zd * zd - dd * (zz - radius * radius);
    if (disc < 0.0) disc = 0.0;
    return pos ? (-zd + sqrt(disc)) / dd : (-zd - sqrt(disc)) / dd;
}

typedef void (*oracle_hv_fn)(const double *v, double *out, void *ctx);

/*
 * CG-Steihaug (Algorithm "Trust-Region CG-Steihaug", after Nocedal and
 * Wright, Alg. 7.2): approximately minimise m(p) = g.p + p.Bp / 2 over
 * |p| <= radius, B given by its products hv.  z_0 = 0, r_0 = g, d_0 = -g;
 * stop when |r_0| < eps (p = 0); per step: on d.Bd <= 0 go to the boundary
 * along d at the root with the smaller m; else alpha = r.r / d.Bd, and if
 * |z + alpha d| >= radius go to the boundary along d (tau >= 0); else
 * r <- r + alpha Bd, stop if |r| < eps, beta = r_new.r_new / r.r,
 * d <- -r + beta d.  The model value m(p) is carried along (m(z + tau d) =
 * m(z) + tau r.d + tau^2 d.Bd / 2, r = g + Bz).  status: 0 residual below
 * eps, 1 boundary, 2 negative curvature, 3 iteration limit.
 */
int oracle_cg_steihaug(int n, const double *g, oracle_hv_fn hv, void *ctx, double radius,
                       double eps, int maxit, double *p, double *m_out, int *iters,
                       int *status)
{
    if (n < 1 || !g || !hv || !p || !(radius > 0.0) || maxit < 0) return ORACLE_EINVAL;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *bd = (double *)malloc(sizeof(double) * (size_t)n);
    if (!r || !d || !bd) { free(r); free(d); free(bd); return ORACLE_EINVAL; }
    for (int i = 0; i < n; ++i) { p[i] = 0.0; r[i] = g[i]; d[i] = -g[i]; }
    double m = 0.0, rr = vdot(n, r, r);
    int st = 3, it = 0;
    if (sqrt(rr) < eps) {
        st = 0;
    } else {
        for (it = 0; it < maxit; ++it) {
            hv(d, bd, ctx);
            double dbd = vdot(n, d, bd), rd = vdot(n, r, d);
            if (dbd <= 0.0) {
                double t1 = to_boundary(n, p, d, radius, 1), t2 = to_boundary(n, p, d, radius, 0);
                double m1 = m + t1 * rd + 0.5 * t1 * t1 * dbd;
                double m2 = m + t2 * rd + 0.5 * t2 * t2 * dbd;
                double t = m1 <= m2 ? t1 : t2;
                for (int i = 0; i < n; ++i) p[i] += t * d[i];
                m = m1 <= m2 ? m1 : m2;
                st = 2; ++it;
                break;
            }
            double alpha = rr / dbd;
            double zn2 = 0.0;
            for (int i = 0; i < n; ++i) { double zi = p[i] + alpha * d[i]; zn2 += zi * zi; }
            if (sqrt(zn2) >= radius) {
                double t = to_boundary(n, p, d, radius, 1);
                for (int i = 0; i < n; ++i) p[i] += t * d[i];
                m += t * rd + 0.5 * t * t * dbd;
                st = 1; ++it;
                break;
            }
            for (int i = 0; i < n; ++i) { p[i] += alpha * d[i]; r[i] += alpha * bd[i]; }
            m += alpha * rd + 0.5 * alpha * alpha * dbd;
            double rr_new = vdot(n, r, r);
            if (sqrt(rr_new) < eps) { st = 0; ++it; break; }
            double beta = rr_new / rr;
            for (int i = 0; i < n; ++i) d[i] = -r[i] + beta * d[i];
            rr = rr_new;
        }
    }
    if (m_out) *m_out = m;
    if (iters) *iters = it;
    if (status) *status = st;
    free(r); free(d); free(bd);
    return ORACLE_OK;
}

typedef struct oracle_hv_ctx {
    int N, d;
    const double *v;      /* the point */
    double delta, h;
    double *tmp, *gp, *gm;
    int products;
} oracle_hv_ctx;

/* B u by a central difference of the exact gradient along u:
 * |u| (grad F(V + h u/|u|) - grad F(V - h u/|u|)) / (2h). */
static void lse_hv(const double *u, double *out, void *vctx)
{
    oracle_hv_ctx *c = (oracle_hv_ctx *)vctx;
    int n = 2 * c->d * c->N;
    double nu = sqrt(vdot(n, u, u));
    if (!(nu > 0.0)) { for (int i = 0; i < n; ++i) out[i] = 0.0; return; }
    double F, s, step = c->h / nu;
    for (int i = 0; i < n; ++i) c->tmp[i] = c->v[i] + step * u[i];
    oracle_lse(c->N, c->d, c->tmp, c->delta, &F, &s, c->gp);
    for (int i = 0; i < n; ++i) c->tmp[i] = c->v[i] - step * u[i];
    oracle_lse(c->N, c->d, c->tmp, c->delta, &F, &s, c->gm);
    for (int i = 0; i < n; ++i) out[i] = (c->gp[i] - c->gm[i]) * (nu / (2.0 * c->h));
    c->products++;
}

/* The product above, for tests. */
int oracle_lse_hv(int N, int d, const double *v, double delta, double h, const double *u,
                  double *out)
{
    if (N < 2 || d < 1 || !v || !u || !out || !(delta > 0.0) || !(h > 0.0))
        return ORACLE_EINVAL;
    size_t n = 2 * (size_t)d * (size_t)N;
    oracle_hv_ctx c = {N, d, v, delta, h, NULL, NULL, NULL, 0};
    c.tmp = (double *)malloc(sizeof(double) * n);
    c.gp = (double *)malloc(sizeof(double) * n);
    c.gm = (double *)malloc(sizeof(double) * n);
    if (!c.tmp || !c.gp || !c.gm) { free(c.tmp); free(c.gp); free(c.gm); return ORACLE_EINVAL; }
    lse_hv(u, out, &c);
    free(c.tmp); free(c.gp); free(c.gm);
    return ORACLE_OK;
}

typedef struct oracle_tr_opts {
    int n_delta;
    double delta[16];     /* the smoothing parameters, stage by stage */
    int max_outer;        /* trust-region iterations per stage */
    int max_cg;           /* CG iterations per step */
    double radius0, radius_max, eta, gtol, fd_step;
    int hessian;          /* 0: B_k = the exact Hessian of F (the paper's model);
                             1: central differences of the gradient with step
                             fd_step (for diagnosis only) */
    int pad;
} oracle_tr_opts;

typedef struct oracle_tr_row {
    int32_t stage, iter;
    double F, s, gnorm, radius, rho, step_norm, pred;
    int32_t cg_iters, cg_status, accepted, pad;
} oracle_tr_row;

int oracle_lse_hv_exact(int N, int d, const double *v, double delta, const double *u,
                        double *out);

/* B u with B the exact Hessian of F_{s,delta} at the context's point
 * (oracle_lse_hv_exact, below). */
static void lse_hv_exact_cb(const double *u, double *out, void *vctx)
{
    oracle_hv_ctx *c = (oracle_hv_ctx *)vctx;
    if (oracle_lse_hv_exact(c->N, c->d, c->v, c->delta, u, out) != ORACLE_OK) {
        int n = 2 * c->d * c->N;
        for (int i = 0; i < n; ++i) out[i] = NAN;
    }
    c->products++;
}

/*
 * The paper's procedure on one frame (Sec. "Optimization procedure";
 * Algorithm "TRSTMI optimization steps", step 2): for each smoothing
 * parameter delta_k in turn, minimise F_{s,delta_k} over the variable V by
 * trust-region iterations whose steps come from CG-Steihaug (above), starting
 * from the previous stage's result.  The model of each step is the paper's
 * m(p) = F + g.p + p.B p / 2 with B the Hessian of F at V (Algorithm
 * "Trust-Region CG-Steihaug", B_k = grad^2 f_k); its products come from
 * oracle_lse_hv_exact, or, with o->hessian = 1, from central differences of
 * the gradient (a diagnosis option).  Per iteration (the standard
 * trust-region loop, Nocedal and Wright Alg. 4.1): g = grad F; stop the
 * stage when |g| <= gtol; p from CG-Steihaug with eps = min(1/2, sqrt|g|) |g|;
 * rho = (F(V) - F(V + p)) / (-m(p)); radius /4 if rho < 1/4, doubled (capped)
 * if rho > 3/4 and |p| reached it; accept if rho > eta, then every column of
 * V is divided by its norm (F does not change).  The radius starts at
 * radius0 in every stage.  v (2dN doubles) is updated in place.
 */
int oracle_tr_solve(int N, int d, double *v, const oracle_tr_opts *o, oracle_tr_row *trace,
                    int cap, int *n_rows)
{
    if (N < 2 || d < 1 || !v || !o || o->n_delta < 1 || o->n_delta > 16) return ORACLE_EINVAL;
    if (o->hessian != 0 && o->hessian != 1) return ORACLE_EINVAL;
    int n = 2 * d * N;
    size_t bytes = sizeof(double) * (size_t)n;
    double *g = (double *)malloc(bytes), *p = (double *)malloc(bytes);
    double *vn = (double *)malloc(bytes);
    oracle_hv_ctx c = {N, d, v, 0.0, o->fd_step, NULL, NULL, NULL, 0};
    c.tmp = (double *)malloc(bytes); c.gp = (double *)malloc(bytes);
    c.gm = (double *)malloc(bytes);
    int st = ORACLE_OK, rows = 0;
    if (!g || !p || !vn || !c.tmp || !c.gp || !c.gm) { st = ORACLE_EINVAL; goto out; }
    st = normalise_columns(N, d, v);
    if (st != ORACLE_OK) goto out;
    for (int k = 0; k < o->n_delta; ++k) {
        double delta = o->delta[k], radius = o->radius0;
        c.delta = delta;
        for (int it = 0; it < o->max_outer; ++it) {
            double F, s, Fn, sn;
            st = oracle_lse(N, d, v, delta, &F, &s, g);
            if (st != ORACLE_OK) goto out;
            double gn = sqrt(vdot(n, g, g));
            if (gn <= o->gtol) break;
            double eps = (sqrt(gn) < 0.5 ? sqrt(gn) : 0.5) * gn, m;
            int cgit, cgst;
            oracle_cg_steihaug(n, g, o->hessian == 1 ? lse_hv : lse_hv_exact_cb, &c, radius, eps,
                               o->max_cg, p, &m, &cgit, &cgst);
            double pn = sqrt(vdot(n, p, p));
            for (int i = 0; i < n; ++i) vn[i] = v[i] + p[i];
            st = oracle_lse(N, d, vn, delta, &Fn, &sn, NULL);
            if (st != ORACLE_OK) goto out;
            double pred = -m;
            double rho = pred > 0.0 ? (F - Fn) / pred : -1.0;
            double r_used = radius;
            if (rho < 0.25) radius *= 0.25;
            else if (rho > 0.75 && pn >= (1.0 - 1e-12) * radius)
                radius = (2.0 * radius < o->radius_max) ? 2.0 * radius : o->radius_max;
            int acc = rho > o->eta;
            if (acc) {
                memcpy(v, vn, bytes);
                st = normalise_columns(N, d, v);
                if (st != ORACLE_OK) goto out;
            }
            if (trace && rows < cap) {
                oracle_tr_row *r = &trace[rows];
                r->stage = k; r->iter = it; r->F = F; r->s = s; r->gnorm = gn;
                r->radius = r_used; r->rho = rho; r->step_norm = pn; r->pred = pred;
                r->cg_iters = cgit; r->cg_status = cgst; r->accepted = acc; r->pad = 0;
            }
            ++rows;
            if (radius < 1e-14) break;
        }
    }
out:
    if (n_rows) *n_rows = rows;
    free(g); free(p); free(vn); free(c.tmp); free(c.gp); free(c.gm);
    return st;
}

/*
 * The exact Hessian of F_{s,delta} at V applied to U, by differentiating the
 * gradient above along U (the chain rule, written out):
 *   d phi_k = (u_k - phi_k Re(phi_k^* u_k)) / r_k,   d r_k = Re(phi_k^* u_k),
 *   dG_jk = d phi_j^* phi_k + phi_j^* d phi_k,        dx_jk = 2 Re(conj(G_jk) dG_jk),
 *   dw_jk = w_jk (dx_jk - sum_l w_l dx_l) / delta     (the shift s cancels),
 *   dM_jk = dw_jk G_jk + w_jk dG_jk                   (j < k; M Hermitian),
 *   dg_k = 2 sum_{j != k} (dM_jk phi_j + M_jk d phi_j),
 *   d rho_k = Re(d phi_k^* g_k + phi_k^* dg_k),
 *   (H u)_k = (dg_k - d phi_k rho_k - phi_k d rho_k) / r_k - grad_k d r_k / r_k.
 * The paper's B_k, used by oracle_tr_solve (its central-difference option,
 * lse_hv, is measured against this function by the tests).
 */
int oracle_lse_hv_exact(int N, int d, const double *v, double delta, const double *u,
                        double *out)
{
    if (N < 2 || d < 1 || !v || !u || !out || !(delta > 0.0)) return ORACLE_EINVAL;
    size_t m = 2 * (size_t)d * (size_t)N, n = (size_t)N * (size_t)(N - 1) / 2;
    double *phi = (double *)malloc(sizeof(double) * m), *dphi = (double *)malloc(sizeof(double) * m);
    double *g = (double *)calloc(m, sizeof(double)), *dg = (double *)calloc(m, sizeof(double));
    double *r = (double *)malloc(sizeof(double) * (size_t)N), *dr = (double *)malloc(sizeof(double) * (size_t)N);
    double *G = (double *)malloc(sizeof(double) * 2 * n), *dG = (double *)malloc(sizeof(double) * 2 * n);
    double *x = (double *)malloc(sizeof(double) * n), *dx = (double *)malloc(sizeof(double) * n);
    int st = ORACLE_OK;
    if (!phi || !dphi || !g || !dg || !r || !dr || !G || !dG || !x || !dx) { st = ORACLE_EINVAL; goto out; }
    for (int k = 0; k < N; ++k) {
        double q = 0.0;
        for (int i = 0; i < d; ++i) {
            double a = v[2 * (k * d + i)], b = v[2 * (k * d + i) + 1];
            q += a * a + b * b;
        }
        if (!(q > 0.0)) { st = ORACLE_EINVAL; goto out; }
        r[k] = sqrt(q);
        double pu = 0.0;   /* Re(phi_k^* u_k) */
        for (int i = 0; i < d; ++i) {
            phi[2 * (k * d + i)] = v[2 * (k * d + i)] / r[k];
            phi[2 * (k * d + i) + 1] = v[2 * (k * d + i) + 1] / r[k];
            pu += phi[2 * (k * d + i)] * u[2 * (k * d + i)] +
                  phi[2 * (k * d + i) + 1] * u[2 * (k * d + i) + 1];
        }
        dr[k] = pu;
        for (int i = 0; i < d; ++i) {
            dphi[2 * (k * d + i)] = (u[2 * (k * d + i)] - phi[2 * (k * d + i)] * pu) / r[k];
            dphi[2 * (k * d + i) + 1] =
                (u[2 * (k * d + i) + 1] - phi[2 * (k * d + i) + 1] * pu) / r[k];
        }
    }
    size_t p = 0;
    double s = 0.0;
    for (int j = 0; j < N; ++j)
        for (int k = j + 1; k < N; ++k, ++p) {
            double gr = 0.0, gi = 0.0, hr = 0.0, hi = 0.0;
            for (int i = 0; i < d; ++i) {
                double a = phi[2 * (j * d + i)], b = phi[2 * (j * d + i) + 1];
                double c = phi[2 * (k * d + i)], e = phi[2 * (k * d + i) + 1];
                double da = dphi[2 * (j * d + i)], db = dphi[2 * (j * d + i) + 1];
                double dc = dphi[2 * (k * d + i)], de = dphi[2 * (k * d + i) + 1];
                gr += a * c + b * e;             /* conj(a + ib)(c + ie) */
                gi += a * e - b * c;
                hr += da * c + db * e + a * dc + b * de;
                hi += da * e - db * c + a * de - b * dc;
            }
            G[2 * p] = gr; G[2 * p + 1] = gi; dG[2 * p] = hr; dG[2 * p + 1] = hi;
            x[p] = gr * gr + gi * gi;
            dx[p] = 2.0 * (gr * hr + gi * hi);
            if (p == 0 || x[p] > s) s = x[p];
        }
    double S = 0.0, T = 0.0;
    for (p = 0; p < n; ++p) S += exp((x[p] - s) / delta);
    for (p = 0; p < n; ++p) T += exp((x[p] - s) / delta) / S * dx[p];
    p = 0;
    for (int j = 0; j < N; ++j)
        for (int k = j + 1; k < N; ++k, ++p) {
            double w = exp((x[p] - s) / delta) / S, dw = w * (dx[p] - T) / delta;
            double Mr = w * G[2 * p], Mi = w * G[2 * p + 1];
            double dMr = dw * G[2 * p] + w * dG[2 * p], dMi = dw * G[2 * p + 1] + w * dG[2 * p + 1];
            for (int i = 0; i < d; ++i) {
                double a = phi[2 * (j * d + i)], b = phi[2 * (j * d + i) + 1];
                double c = phi[2 * (k * d + i)], e = phi[2 * (k * d + i) + 1];
                double da = dphi[2 * (j * d + i)], db = dphi[2 * (j * d + i) + 1];
                double dc = dphi[2 * (k * d + i)], de = dphi[2 * (k * d + i) + 1];
                /* column k: M phi_j, dM phi_j + M dphi_j */
                g[2 * (k * d + i)] += 2.0 * (Mr * a - Mi * b);
                g[2 * (k * d + i) + 1] += 2.0 * (Mr * b + Mi * a);
                dg[2 * (k * d + i)] += 2.0 * (dMr * a - dMi * b + Mr * da - Mi * db);
                dg[2 * (k * d + i) + 1] += 2.0 * (dMr * b + dMi * a + Mr * db + Mi * da);
                /* column j: conj(M) phi_k, conj(dM) phi_k + conj(M) dphi_k */
                g[2 * (j * d + i)] += 2.0 * (Mr * c + Mi * e);
                g[2 * (j * d + i) + 1] += 2.0 * (Mr * e - Mi * c);
                dg[2 * (j * d + i)] += 2.0 * (dMr * c + dMi * e + Mr * dc + Mi * de);
                dg[2 * (j * d + i) + 1] += 2.0 * (dMr * e - dMi * c + Mr * de - Mi * dc);
            }
        }
    for (int k = 0; k < N; ++k) {
        double rho = 0.0, drho = 0.0;
        for (int i = 0; i < d; ++i) {
            size_t a = 2 * ((size_t)k * d + i);
            rho += phi[a] * g[a] + phi[a + 1] * g[a + 1];
            drho += dphi[a] * g[a] + dphi[a + 1] * g[a + 1] + phi[a] * dg[a] + phi[a + 1] * dg[a + 1];
        }
        for (int i = 0; i < d; ++i) {
            size_t a = 2 * ((size_t)k * d + i);
            for (int c = 0; c < 2; ++c) {
                double grad = (g[a + c] - phi[a + c] * rho) / r[k];
                out[a + c] = (dg[a + c] - dphi[a + c] * rho - phi[a + c] * drho) / r[k] -
                             grad * dr[k] / r[k];
            }
        }
    }
out:
    free(phi); free(dphi); free(g); free(dg); free(r); free(dr); free(G); free(dG); free(x); free(dx);
    return st;
}
