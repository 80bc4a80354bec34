/*
 * FP64 CPU oracle for one Vegas iteration and its grid refinement.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists so that the CUDA path can be
 * checked against a plain, slow, obviously correct restatement of the method.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * build, load or call it; the product library never does, and this file
 * includes nothing from it (no shared headers, helpers or constants).
 *
 * What is computed, step by step (VegasFlow, Sec. 2.2 "Integration
 * algorithms": a per-event step that draws random numbers and an
 * after-iteration step that refines how they are drawn; the Vegas method
 * itself is the one the paper cites in Sec. 1 and Sec. 2.2, Lepage 1978/1980):
 *
 *   1. counter-based Philox4x32-10 words per sample          (oracle_philox4x32_10)
 *   2. integer split of a word into bin j and fraction        (oracle_map_sample)
 *   3. the adaptive-grid change of variables x(y), J(y)       (oracle_map_sample)
 *   4. the integrand: Lepage Gaussian of Eq. 1, its two-peak
 *      mixture, the constant function, Genz Eq. 2 and Eq. 3  (oracle_integrand)
 *   5. per-iteration sums S1 = sum fJ, S2 = sum (fJ)^2        (oracle_iterate)
 *   6. per-dimension per-bin histogram of (fJ)^2              (oracle_iterate)
 *   7. smoothing, damping and equal-weight re-partition       (oracle_refine)
 *   8. inverse-variance combination of iterations             (oracle_combine)
 *   9. gradient of the fixed-grid Eq. 1 estimate with respect
 *      to (mu, a), over the same samples                      (oracle_gauss_gradient)
 *
 * Every floating-point quantity is double; sums are carried in long double so
 * that the oracle's own rounding is far below the parity tolerance.  The file
 * is compiled with -ffp-contract=off so that no multiply-add is fused.
 *
 * Pins (in the CPU test suite): Philox words against an independent library
 * implementation; the identity map on a uniform grid; exact results for the
 * constant integrand; closed-form Gaussian integrals; brute-force quadrature
 * at d <= 2; refinement invariants; hand-worked combination examples; for the
 * gradient, central finite differences of the estimator and the analytic erf
 * derivatives of the integral.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_DIM 64

/* ------------------------------------------------------------------------- */
/* 1. Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random       */
/*    numbers: as easy as 1, 2, 3", Sec. 5: the Philox-4x32 bijection).        */
/* ------------------------------------------------------------------------- */

/* Multipliers of the two 32x32->64 products of one round. */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
/* Weyl increments of the key schedule (golden ratio, sqrt(3)-1). */
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

/* One Philox-4x32 round: the two products split into (hi, lo) halves; the high
 * halves are xored with the other two counter words and the round key, and the
 * words are permuted. */
static void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ c[1] ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ c[3] ^ k1;
    uint32_t y3 = lo0;
    c[0] = y0; c[1] = y1; c[2] = y2; c[3] = y3;
}

/* Ten rounds; round r uses the key (k0 + r*W0, k1 + r*W1) mod 2^32. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k0, k1);
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Batch form for the tests: ctrs is n x 4, out is n x 4. */
void oracle_philox_batch(uint64_t n, const uint32_t *ctrs, const uint32_t key[2], uint32_t *out)
{
    for (uint64_t i = 0; i < n; ++i)
        oracle_philox4x32_10(ctrs + 4 * i, key, out + 4 * i);
}

/* The counter of one sample's q-th Philox call.  Key = the 64-bit seed (low word
 * first).  Counter = (sample index low, sample index high, q | integral<<8,
 * iteration).  The iteration and the dimension block sit in the spare words so
 * that iterations and dimension blocks draw independent streams. */
void oracle_sample_counter(uint64_t i, uint32_t q, uint32_t integral_id, uint32_t iter,
                           uint32_t ctr[4])
{
    ctr[0] = (uint32_t)i;
    ctr[1] = (uint32_t)(i >> 32);
    ctr[2] = q | (integral_id << 8);
    ctr[3] = iter;
}

/* Words of one sample: dimension k takes word k mod 4 of call q = floor(k/4). */
void oracle_sample_words(uint64_t seed, uint32_t integral_id, uint32_t iter, uint64_t i,
                         int dim, uint32_t *words)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int ncalls = (dim + 3) / 4;
    for (int q = 0; q < ncalls; ++q) {
        uint32_t ctr[4], out[4];
        oracle_sample_counter(i, (uint32_t)q, integral_id, iter, ctr);
        oracle_philox4x32_10(ctr, key, out);
        for (int w = 0; w < 4 && 4 * q + w < dim; ++w)
            words[4 * q + w] = out[w];
    }
}

/* ------------------------------------------------------------------------- */
/* 2-3. Bin, fraction and the grid map (Lepage 1978, Sec. 2: a piecewise-      */
/*      linear map whose N bins each carry probability 1/N).                   */
/* ------------------------------------------------------------------------- */

/* edges: dim rows of N+1 increasing values, e[k][0] = 0, e[k][N] = 1.
 * For word w: t = w*N (64-bit); bin j = t >> 32 in [0, N-1]; the low 32 bits
 * l give the position inside the bin, frac = (l + 1/2) 2^-32 in (0, 1).
 * x_k = e_j + frac * (e_{j+1} - e_j); J = prod_k N (e_{j+1} - e_j). */
void oracle_map_sample(int dim, int nbins, const double *edges, const uint32_t *words,
                       double *x, double *jac, int32_t *bins)
{
    double J = 1.0;
    for (int k = 0; k < dim; ++k) {
        const double *e = edges + (size_t)k * (nbins + 1);
        uint64_t t = (uint64_t)words[k] * (uint64_t)nbins;
        uint32_t j = (uint32_t)(t >> 32);
        uint32_t l = (uint32_t)t;
        double frac = ((double)l + 0.5) * 0x1p-32;
        double width = e[j + 1] - e[j];
        x[k] = e[j] + frac * width;
        J = J * ((double)nbins * width);
        if (bins) bins[k] = (int32_t)j;
    }
    *jac = J;
}

/* ------------------------------------------------------------------------- */
/* 4. Integrands over [0,1]^d (VegasFlow Sec. 3.1).                            */
/* ------------------------------------------------------------------------- */

enum {
    ORACLE_GAUSS = 0,      /* Eq. 1: params [a, mu_1..mu_d]                      */
    ORACLE_GAUSS_MIX2 = 1, /* (G(x;muA,a) + G(x;muB,a))/2: [a, muA_1..d, muB_1..d]*/
    ORACLE_FLAT = 2,       /* f = 1: no params                                   */
    ORACLE_GENZ_DISC = 3,  /* Eq. 2: params [a_1..a_d, c_1..c_d]                 */
    ORACLE_GENZ_PPEAK = 4  /* Eq. 3: params [a_1..a_d, c_1..c_d]                 */
};

/* Normalisation of Eq. 1 as used here: each factor exp(-(x-mu)^2/a^2)/(a sqrt(pi))
 * integrates to 1 over the real line, so the [0,1]^d integral is
 * prod_k (erf((1-mu_k)/a) + erf(mu_k/a))/2. */
static double gauss_product(int dim, double a, const double *mu, const double *x)
{
    double s = 0.0;
    for (int k = 0; k < dim; ++k) {
        double u = x[k] - mu[k];
        s += u * u;
    }
    double norm = pow(a * sqrt(M_PI), -(double)dim);
    return norm * exp(-s / (a * a));
}

/* Eq. 2 normalised to integrate to 1 over [0,1]^d:
 * 0 if any x_k <= a_k, else exp(sum c_k x_k) / prod_k (e^{c_k} - e^{c_k a_k}) / c_k. */
static double genz_disc(int dim, const double *p, const double *x)
{
    const double *a = p, *c = p + dim;
    double s = 0.0, norm = 1.0;
    for (int k = 0; k < dim; ++k) {
        if (x[k] <= a[k]) return 0.0;
        s += c[k] * x[k];
        norm *= (exp(c[k]) - exp(c[k] * a[k])) / c[k];
    }
    return exp(s) / norm;
}

/* Eq. 3 normalised to integrate to 1 over [0,1]^d: each factor
 * 1/(c^-2 + (x-a)^2) integrates to c (atan(c(1-a)) + atan(c a)). */
static double genz_ppeak(int dim, const double *p, const double *x)
{
    const double *a = p, *c = p + dim;
    double v = 1.0;
    for (int k = 0; k < dim; ++k) {
        double u = x[k] - a[k];
        double factor = 1.0 / (1.0 / (c[k] * c[k]) + u * u);
        double integral = c[k] * (atan(c[k] * (1.0 - a[k])) + atan(c[k] * a[k]));
        v *= factor / integral;
    }
    return v;
}

double oracle_integrand(int id, int dim, const double *params, const double *x)
{
    switch (id) {
    case ORACLE_GAUSS:
        return gauss_product(dim, params[0], params + 1, x);
    case ORACLE_GAUSS_MIX2:
        return 0.5 * (gauss_product(dim, params[0], params + 1, x) +
                      gauss_product(dim, params[0], params + 1 + dim, x));
    case ORACLE_FLAT:
        return 1.0;
    case ORACLE_GENZ_DISC:
        return genz_disc(dim, params, x);
    case ORACLE_GENZ_PPEAK:
        return genz_ppeak(dim, params, x);
    default:
        return NAN;
    }
}

/* ------------------------------------------------------------------------- */
/* 5-6. One iteration: n samples, their sums and the refinement histogram.     */
/* ------------------------------------------------------------------------- */

typedef struct {
    int dim, nbins, integrand, adapt;
    const double *edges, *params;
    const double *box_lo, *box_w; /* integration box (NULL: the unit cube) */
    uint64_t seed, begin, end;
    uint32_t integral_id, iter;
    long double s1, s2;
    long double *hist; /* dim * nbins, this slice's own */
    uint64_t nonfinite;
} slice_job;

static void *run_slice(void *arg)
{
    slice_job *jb = (slice_job *)arg;
    uint32_t words[ORACLE_MAX_DIM];
    double x[ORACLE_MAX_DIM];
    int32_t bins[ORACLE_MAX_DIM];
    for (uint64_t i = jb->begin; i < jb->end; ++i) {
        double J;
        oracle_sample_words(jb->seed, jb->integral_id, jb->iter, i, jb->dim, words);
        oracle_map_sample(jb->dim, jb->nbins, jb->edges, words, x, &J, bins);
        if (jb->box_lo) /* the box [lo, lo + w]: x = lo + w u, dx = (prod w) du */
            for (int k = 0; k < jb->dim; ++k) {
                x[k] = jb->box_lo[k] + jb->box_w[k] * x[k];
                J *= jb->box_w[k];
            }
        double fw = oracle_integrand(jb->integrand, jb->dim, jb->params, x) * J;
        if (!isfinite(fw)) {
            jb->nonfinite++;
            continue;
        }
        double fw2 = fw * fw;
        jb->s1 += fw;
        jb->s2 += fw2;
        if (jb->adapt)
            for (int k = 0; k < jb->dim; ++k)
                jb->hist[(size_t)k * jb->nbins + bins[k]] += fw2;
    }
    return NULL;
}

/* One Vegas iteration over sample indices [first, first + n) (the whole
 * iteration when first = 0 and n is its sample count; a shard otherwise), over
 * the box [lo, lo + w] (box_lo, box_w: dim doubles each; NULL: the unit cube --
 * the grid stays in unit coordinates u and the integrand sees x = lo + w u with
 * the Jacobian's extra factor prod w).  Outputs the sums S1, S2, the
 * count of non-finite f*J values (left out of the sums), and, when adapt != 0,
 * adds the histogram sum over samples of (fJ)^2 per (dimension, bin) into hist
 * (dim * nbins doubles, caller-initialised).  The index range is cut into
 * nthreads contiguous slices whose sums are added in slice order.
 * Returns 0, or -1 on invalid arguments. */
int oracle_iterate_range_box(int dim, int nbins, const double *edges, uint64_t seed,
                             uint32_t integral_id, uint32_t iter, uint64_t first, uint64_t n,
                             int integrand, const double *params, const double *box_lo,
                             const double *box_w, int adapt, int nthreads, double *S1,
                             double *S2, double *hist, uint64_t *nonfinite)
{
    if (dim < 1 || dim > ORACLE_MAX_DIM || nbins < 1 || nthreads < 1) return -1;
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > n && n > 0) nthreads = (int)n;
    if (n == 0) nthreads = 1;
    slice_job *jobs = calloc((size_t)nthreads, sizeof(slice_job));
    pthread_t *tids = calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tids) { free(jobs); free(tids); return -1; }
    for (int t = 0; t < nthreads; ++t) {
        slice_job *jb = &jobs[t];
        jb->dim = dim; jb->nbins = nbins; jb->integrand = integrand; jb->adapt = adapt;
        jb->edges = edges; jb->params = params; jb->seed = seed;
        jb->box_lo = box_lo; jb->box_w = box_w;
        jb->integral_id = integral_id; jb->iter = iter;
        /* slice t is [floor(n t / T), floor(n (t+1) / T)) */
        jb->begin = first + (uint64_t)(((unsigned __int128)n * (uint64_t)t) / (uint64_t)nthreads);
        jb->end = first + (uint64_t)(((unsigned __int128)n * (uint64_t)(t + 1)) / (uint64_t)nthreads);
        jb->hist = adapt ? calloc((size_t)dim * nbins, sizeof(long double)) : NULL;
    }
    if (nthreads == 1) {
        run_slice(&jobs[0]);
    } else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&tids[t], NULL, run_slice, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) pthread_join(tids[t], NULL);
    }
    long double s1 = 0, s2 = 0;
    uint64_t bad = 0;
    for (int t = 0; t < nthreads; ++t) {
        s1 += jobs[t].s1;
        s2 += jobs[t].s2;
        bad += jobs[t].nonfinite;
    }
    if (adapt) {
        for (size_t b = 0; b < (size_t)dim * nbins; ++b) {
            long double h = 0;
            for (int t = 0; t < nthreads; ++t) h += jobs[t].hist[b];
            hist[b] += (double)h;
        }
        for (int t = 0; t < nthreads; ++t) free(jobs[t].hist);
    }
    *S1 = (double)s1;
    *S2 = (double)s2;
    *nonfinite = bad;
    free(jobs);
    free(tids);
    return 0;
}

int oracle_iterate_range(int dim, int nbins, const double *edges, uint64_t seed,
                         uint32_t integral_id, uint32_t iter, uint64_t first, uint64_t n,
                         int integrand, const double *params, int adapt, int nthreads,
                         double *S1, double *S2, double *hist, uint64_t *nonfinite)
{
    return oracle_iterate_range_box(dim, nbins, edges, seed, integral_id, iter, first, n,
                                    integrand, params, NULL, NULL, adapt, nthreads, S1, S2, hist,
                                    nonfinite);
}

int oracle_iterate(int dim, int nbins, const double *edges, uint64_t seed, uint32_t integral_id,
                   uint32_t iter, uint64_t n, int integrand, const double *params, int adapt,
                   int nthreads, double *S1, double *S2, double *hist, uint64_t *nonfinite)
{
    return oracle_iterate_range(dim, nbins, edges, seed, integral_id, iter, 0, n, integrand,
                                params, adapt, nthreads, S1, S2, hist, nonfinite);
}

/* Estimate of one iteration from its sums: I = S1/n and the unbiased variance
 * of the mean, (S2/n - I^2)/(n-1), clamped at 0 against rounding. */
void oracle_estimate(double S1, double S2, uint64_t n, double *I, double *var)
{
    double nn = (double)n;
    *I = S1 / nn;
    double v = (S2 / nn - (*I) * (*I)) / (nn - 1.0);
    *var = v > 0.0 ? v : 0.0;
}

/* ------------------------------------------------------------------------- */
/* 7. Grid refinement (Lepage 1978 Sec. 3; smoothing of Lepage 1980).          */
/* ------------------------------------------------------------------------- */

/* Damping of one normalised bin weight r in [0,1]: ((r - 1)/ln r)^alpha,
 * with the limits 0 at r = 0 and 1 at r = 1. */
double oracle_damp(double r, double alpha)
{
    if (r <= 0.0) return 0.0;
    if (r == 1.0) return 1.0;
    return pow((r - 1.0) / log(r), alpha);
}

/* Three-point smoothing of one histogram row (nbins >= 2): interior bins take
 * the mean of themselves and both neighbours, the two end bins the mean of
 * themselves and their one neighbour. */
void oracle_smooth(int nbins, const double *hist, double *out)
{
    int N = nbins;
    out[0] = (hist[0] + hist[1]) / 2.0;
    for (int j = 1; j < N - 1; ++j) out[j] = (hist[j - 1] + hist[j] + hist[j + 1]) / 3.0;
    out[N - 1] = (hist[N - 2] + hist[N - 1]) / 2.0;
}

/* Refine one dimension in place.  hist: the nbins (fJ)^2 sums of the dimension;
 * e: its nbins+1 edges.  Returns 1 if refined, 0 if skipped (nbins < 2, or a
 * zero or non-finite histogram). */
int oracle_refine_dim(int nbins, double *e, const double *hist, double alpha)
{
    int N = nbins;
    if (N < 2) return 0;
    double total = 0.0;
    for (int j = 0; j < N; ++j) total += hist[j];
    if (!(total > 0.0) || !isfinite(total)) return 0;

    double *sm = malloc(sizeof(double) * N);
    double *m = malloc(sizeof(double) * N);
    double *C = malloc(sizeof(double) * (N + 1));
    double *old = malloc(sizeof(double) * (N + 1));
    memcpy(old, e, sizeof(double) * (N + 1));

    oracle_smooth(N, hist, sm);

    double smsum = 0.0;
    for (int j = 0; j < N; ++j) smsum += sm[j];

    /* normalise, damp */
    for (int j = 0; j < N; ++j) m[j] = oracle_damp(sm[j] / smsum, alpha);

    /* cumulative weight at the old edges */
    C[0] = 0.0;
    for (int j = 0; j < N; ++j) C[j + 1] = C[j] + m[j];
    double delta = C[N] / N;

    /* new edge l sits where the piecewise-linear cumulative weight reaches l*delta:
     * in the old bin b with C[b] < l*delta <= C[b+1] */
    int b = 0;
    for (int l = 1; l < N; ++l) {
        double target = l * delta;
        while (b < N - 1 && !(target <= C[b + 1])) ++b;
        double width = old[b + 1] - old[b];
        e[l] = old[b] + (target - C[b]) / m[b] * width;
    }
    e[0] = old[0];
    e[N] = old[N];

    free(sm); free(m); free(C); free(old);
    return 1;
}

/* Refine every dimension: edges is dim x (nbins+1), hist is dim x nbins.
 * Returns the number of dimensions refined. */
int oracle_refine(int dim, int nbins, double *edges, const double *hist, double alpha)
{
    int refined = 0;
    for (int k = 0; k < dim; ++k)
        refined += oracle_refine_dim(nbins, edges + (size_t)k * (nbins + 1),
                                     hist + (size_t)k * nbins, alpha);
    return refined;
}

/* ------------------------------------------------------------------------- */
/* 8. Combination of iterations (Lepage 1978 Sec. 2: the cumulative estimate  */
/*    is the inverse-variance weighted mean, with its chi^2 per d.o.f.).       */
/* ------------------------------------------------------------------------- */

void oracle_combine(int K, const double *I, const double *var, double *mean, double *sigma,
                    double *chi2_dof)
{
    if (K <= 0) { *mean = NAN; *sigma = NAN; *chi2_dof = NAN; return; }
    int any_zero = 0;
    for (int k = 0; k < K; ++k) if (!(var[k] > 0.0)) any_zero = 1;
    if (any_zero) {
        /* some iteration has no spread at all: plain mean, zero error */
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += I[k];
        *mean = s / K;
        *sigma = 0.0;
        double c = 0.0;
        for (int k = 0; k < K; ++k) c += (I[k] - *mean) * (I[k] - *mean);
        *chi2_dof = (K > 1 && c == 0.0) ? 0.0 : (K > 1 ? INFINITY : 0.0);
        return;
    }
    double wsum = 0.0, wisum = 0.0;
    for (int k = 0; k < K; ++k) {
        wsum += 1.0 / var[k];
        wisum += I[k] / var[k];
    }
    *mean = wisum / wsum;
    *sigma = sqrt(1.0 / wsum);
    double chi2 = 0.0;
    for (int k = 0; k < K; ++k) chi2 += (I[k] - *mean) * (I[k] - *mean) / var[k];
    *chi2_dof = K > 1 ? chi2 / (K - 1) : 0.0;
}

/* Uniform starting grid: e[k][l] = l/N. */
void oracle_uniform_grid(int dim, int nbins, double *edges)
{
    for (int k = 0; k < dim; ++k)
        for (int l = 0; l <= nbins; ++l)
            edges[(size_t)k * (nbins + 1) + l] = (double)l / nbins;
}

/* Batch forms for the tests (one call per array instead of per sample). */
void oracle_map_batch(uint64_t n, int dim, int nbins, const double *edges, const uint32_t *words,
                      double *x, double *jac, int32_t *bins)
{
    for (uint64_t i = 0; i < n; ++i)
        oracle_map_sample(dim, nbins, edges, words + i * dim, x + i * dim, jac + i,
                          bins ? bins + i * dim : NULL);
}

void oracle_integrand_batch(uint64_t n, int id, int dim, const double *params, const double *x,
                            double *f)
{
    for (uint64_t i = 0; i < n; ++i) f[i] = oracle_integrand(id, dim, params, x + i * dim);
}

/* ------------------------------------------------------------------------- */
/* Gradient of the fixed-grid estimator of Eq. 1 with respect to its          */
/* parameters.  On a fixed grid the samples do not depend on the parameters,  */
/* so d/dtheta of (1/n) sum_i f(x_i) J_i is (1/n) sum_i J_i df/dtheta(x_i).    */
/* For f = (a sqrt(pi))^-d exp(-sum_k (x_k - mu_k)^2 / a^2):                    */
/*   df/dmu_k = f * 2 (x_k - mu_k) / a^2                                         */
/*   df/da    = f * (2 sum_k (x_k - mu_k)^2 / a^3 - d / a)                        */
/* params = [a, mu_1..mu_d].  out: [I, dI/dmu_1..dI/dmu_d, dI/da] then the      */
/* variances of those d+2 sample means, then the non-finite count.  box_lo,     */
/* box_w: the integration box as in oracle_iterate_range_box (NULL: unit cube). */
/* ------------------------------------------------------------------------- */
int oracle_gauss_gradient_box(int dim, int nbins, const double *edges, uint64_t seed,
                              uint32_t iter, uint64_t n, const double *params,
                              const double *box_lo, const double *box_w, double *out)
{
    if (dim < 1 || dim > ORACLE_MAX_DIM || n < 2) return -1;
    const int nc = dim + 2;
    long double *s1 = calloc((size_t)nc, sizeof(long double));
    long double *s2 = calloc((size_t)nc, sizeof(long double));
    double *g = malloc(sizeof(double) * nc);
    if (!s1 || !s2 || !g) { free(s1); free(s2); free(g); return -1; }
    const double a = params[0];
    const double *mu = params + 1;
    uint32_t words[ORACLE_MAX_DIM];
    double x[ORACLE_MAX_DIM];
    uint64_t bad = 0;
    for (uint64_t i = 0; i < n; ++i) {
        double J;
        oracle_sample_words(seed, 0, iter, i, dim, words);
        oracle_map_sample(dim, nbins, edges, words, x, &J, NULL);
        if (box_lo) /* as in the iteration: x = lo + w u, J gains prod w */
            for (int k = 0; k < dim; ++k) {
                x[k] = box_lo[k] + box_w[k] * x[k];
                J *= box_w[k];
            }
        double fw = gauss_product(dim, a, mu, x) * J;
        if (!isfinite(fw)) { bad++; continue; }
        double sq = 0.0;
        g[0] = fw;
        for (int k = 0; k < dim; ++k) {
            double u = x[k] - mu[k];
            g[1 + k] = fw * 2.0 * u / (a * a);
            sq += u * u;
        }
        g[dim + 1] = fw * (2.0 * sq / (a * a * a) - dim / a);
        for (int c = 0; c < nc; ++c) {
            s1[c] += g[c];
            s2[c] += (long double)g[c] * g[c];
        }
    }
    for (int c = 0; c < nc; ++c) {
        long double m = s1[c] / (long double)n;
        long double v = (s2[c] / (long double)n - m * m) / (long double)(n - 1);
        out[c] = (double)m;
        out[nc + c] = v > 0 ? (double)v : 0.0;
    }
    out[2 * nc] = (double)bad;
    free(s1); free(s2); free(g);
    return 0;
}

int oracle_gauss_gradient(int dim, int nbins, const double *edges, uint64_t seed, uint32_t iter,
                          uint64_t n, const double *params, double *out)
{
    return oracle_gauss_gradient_box(dim, nbins, edges, seed, iter, n, params, NULL, NULL, out);
}
