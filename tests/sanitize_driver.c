/* Host code under AddressSanitizer and UndefinedBehaviorSanitizer: the FP64
 * oracle (every integrand, adapting iterations on several threads, refinement,
 * combination, the Gaussian gradient) and the C ABI's host-side paths that need
 * no GPU (workspace sizes, argument checks, checkpoint blob validation, error
 * strings).  Built and run by tests/test_sanitizers.py; exits 0 when every
 * check holds and the sanitizers report nothing.  With -DORACLE_ONLY (the
 * ThreadSanitizer build, which the CUDA runtime does not support) only the
 * oracle part runs. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "vegas.h"

/* the oracle's entry points (oracle/vegas_oracle.c, linked in) */
void oracle_uniform_grid(int dim, int nbins, double *edges);
int oracle_iterate(int dim, int nbins, const double *edges, uint64_t seed, uint32_t integral_id,
                   uint32_t iter, uint64_t n, int integrand, const double *params, int adapt,
                   int nthreads, double *S1, double *S2, double *hist, uint64_t *nonfinite);
void oracle_estimate(double S1, double S2, uint64_t n, double *I, double *var);
int oracle_refine(int dim, int nbins, double *edges, const double *hist, double alpha);
void oracle_combine(int K, const double *I, const double *var, double *mean, double *sigma,
                    double *chi2_dof);
int oracle_gauss_gradient(int dim, int nbins, const double *edges, uint64_t seed, uint32_t iter,
                          uint64_t n, const double *params, double *out);

static int failures = 0;
#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            fprintf(stderr, "check failed: %s (line %d)\n", #cond, __LINE__); \
            ++failures;                                               \
        }                                                             \
    } while (0)

static void oracle_runs(void) {
    enum { D = 5, N = 9, K = 4 };
    double params[1 + 2 * D];
    for (int id = 0; id <= 4; ++id) {
        /* parameters valid for every integrand: a / c > 0, centres inside */
        params[0] = 0.3;
        for (int k = 0; k < 2 * D; ++k) params[1 + k] = 0.2 + 0.05 * k;
        double *p = params;
        double alt[2 * D];
        if (id == 3 || id == 4) { /* Genz: [a_1..a_d, c_1..c_d] */
            for (int k = 0; k < D; ++k) { alt[k] = 0.1 + 0.1 * k; alt[D + k] = 2.0 + k; }
            p = alt;
        }
        double *edges = malloc(sizeof(double) * D * (N + 1));
        double *hist = malloc(sizeof(double) * D * N);
        double I[K], var[K];
        oracle_uniform_grid(D, N, edges);
        for (int t = 0; t < K; ++t) {
            double S1 = 0, S2 = 0;
            uint64_t bad = 0;
            CHECK(oracle_iterate(D, N, edges, 7, 0, (uint32_t)t, 3001, id, p, 1, 3, &S1, &S2, hist,
                                 &bad) == 0);
            oracle_estimate(S1, S2, 3001, &I[t], &var[t]);
            CHECK(isfinite(I[t]) && var[t] >= 0.0);
            CHECK(oracle_refine(D, N, edges, hist, 1.5) == D);  /* every row refined */
            for (int k = 0; k < D; ++k)
                for (int l = 0; l < N; ++l) CHECK(edges[k * (N + 1) + l + 1] > edges[k * (N + 1) + l]);
        }
        double mean, sigma, chi2;
        oracle_combine(K, I, var, &mean, &sigma, &chi2);
        CHECK(isfinite(mean));
        free(edges);
        free(hist);
    }
    double edges[3 * 11];
    double out[2 * (3 + 2) + 1];
    const double gp[4] = {0.2, 0.4, 0.5, 0.6};
    oracle_uniform_grid(3, 10, edges);
    CHECK(oracle_gauss_gradient(3, 10, edges, 5, 0, 2000, gp, out) == 0);
}

#ifndef ORACLE_ONLY
static void capi_host_paths(void) {
    size_t bytes = 0;
    CHECK(vegas_workspace_bytes(8, 50, 16, &bytes) == VEGAS_OK && bytes > 0);
    CHECK(vegas_workspace_bytes(0, 50, 16, &bytes) == VEGAS_EINVAL);
    CHECK(vegas_workspace_bytes(VEGAS_MAX_DIM + 1, 50, 16, &bytes) == VEGAS_EINVAL);
    CHECK(vegas_workspace_bytes(8, VEGAS_MAX_BINS + 1, 16, &bytes) == VEGAS_EINVAL);
    CHECK(vegas_workspace_bytes(8, 50, 16, NULL) == VEGAS_EINVAL);

    vegas_state *s = (vegas_state *)0x1;
    const double p[5] = {0.1, 0.5, 0.5, 0.5, 0.5};
    CHECK(vegas_init_grid(&s, 4, 50, 1, VEGAS_FP64, VEGAS_GAUSS, p, 5, 8, NULL, bytes, NULL) ==
          VEGAS_EINVAL);
    CHECK(s == NULL);
    CHECK(vegas_init_grid(NULL, 4, 50, 1, VEGAS_FP64, VEGAS_GAUSS, p, 5, 8, NULL, bytes, NULL) ==
          VEGAS_EINVAL);
    CHECK(vegas_init_grid(&s, 4, 50, 1, 7, VEGAS_GAUSS, p, 5, 8, (void *)0x10000, bytes, NULL) ==
          VEGAS_EINVAL);
    CHECK(vegas_destroy(NULL) == VEGAS_OK);
    CHECK(vegas_iterate(NULL, 1000, 1) == VEGAS_EINVAL);
    CHECK(vegas_refine(NULL, 1.5) == VEGAS_EINVAL);
    CHECK(vegas_set_user_integrand(NULL, NULL, NULL) == VEGAS_EINVAL);
    CHECK(vegas_shard_export(NULL, NULL) == VEGAS_EINVAL);
    CHECK(vegas_shard_import(NULL, NULL, 10) == VEGAS_EINVAL);
    CHECK(vegas_shard_export_rows(NULL, 0, 1, NULL) == VEGAS_EINVAL);
    CHECK(vegas_shard_import_rows(NULL, 0, 1, NULL, 10) == VEGAS_EINVAL);
    CHECK(vegas_grid_digest(NULL, NULL) == VEGAS_EINVAL);

    /* checkpoint blobs: wrong magic, truncated header, truncated body */
    unsigned char blob[512];
    memset(blob, 0, sizeof(blob));
    memcpy(blob, "NOTVEGAS", 8);
    CHECK(vegas_import_state(&s, blob, sizeof(blob), NULL, 0, NULL) == VEGAS_EINVAL);
    memcpy(blob, "VEGASB3\0", 8);
    CHECK(vegas_import_state(&s, blob, 24, NULL, 0, NULL) == VEGAS_EINVAL);
    CHECK(vegas_import_state(&s, blob, sizeof(blob), NULL, 0, NULL) == VEGAS_EINVAL);
    CHECK(vegas_import_state(&s, NULL, 0, NULL, 0, NULL) == VEGAS_EINVAL);

    size_t bb = 0;
    const int dims[2] = {2, 40};
    const uint64_t ns[2] = {1000, 1000};
    CHECK(vegas_batch_workspace_bytes(2, dims, ns, 50, 4, &bb) == VEGAS_EINVAL);

    for (int st = -1; st <= 8; ++st) {
        const char *m = vegas_strerror(st);
        CHECK(m != NULL && strlen(m) > 0);
    }
}
#endif

int main(void) {
    oracle_runs();
#ifndef ORACLE_ONLY
    capi_host_paths();
#endif
    if (failures) {
        fprintf(stderr, "%d checks failed\n", failures);
        return 1;
    }
    printf("sanitized host paths: ok\n");
    return 0;
}
