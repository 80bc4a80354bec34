/* The C ABI used from a plain C program, with no Python in the process: the
 * caller allocates the workspace with cudaMalloc, creates its own stream, runs
 * a Vegas schedule on the d-dimensional Eq. 1 Gaussian and reads the result.
 * Built (gcc, CUDA runtime) and run by tests/test_gpu_capi_driver.py.
 *
 *   capi_driver MODE SEED DIM NBINS A N_ADAPT K_ADAPT N_FIXED K_FIXED
 *
 * prints one line "I_0 ... I_{K-1}" (every iteration's estimate) and one line
 * "mean sigma chi2_dof n_iter"; exits 1 with the status text on any error. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "vegas.h"

#define CALL(x)                                                                        \
    do {                                                                               \
        int rc_ = (x);                                                                 \
        if (rc_ != VEGAS_OK) {                                                         \
            fprintf(stderr, "%s failed: %s\n", #x, vegas_strerror(rc_));               \
            return 1;                                                                  \
        }                                                                              \
    } while (0)

#define CUDA(x)                                                                        \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            fprintf(stderr, "%s failed: %s\n", #x, cudaGetErrorString(e_));            \
            return 1;                                                                  \
        }                                                                              \
    } while (0)

int main(int argc, char **argv) {
    if (argc != 10) {
        fprintf(stderr, "usage: %s MODE SEED DIM NBINS A N_ADAPT K_ADAPT N_FIXED K_FIXED\n",
                argv[0]);
        return 2;
    }
    const int mode = atoi(argv[1]);
    const uint64_t seed = strtoull(argv[2], NULL, 10);
    const int dim = atoi(argv[3]), nbins = atoi(argv[4]);
    const double a = atof(argv[5]);
    const uint64_t n_adapt = strtoull(argv[6], NULL, 10);
    const int k_adapt = atoi(argv[7]);
    const uint64_t n_fixed = strtoull(argv[8], NULL, 10);
    const int k_fixed = atoi(argv[9]);
    if (dim < 1 || dim > VEGAS_MAX_DIM || k_adapt < 0 || k_fixed < 0 || k_adapt + k_fixed < 1)
        return 2;
    const int iters = k_adapt + k_fixed;

    double params[1 + VEGAS_MAX_DIM];
    params[0] = a;
    for (int k = 0; k < dim; ++k) params[1 + k] = 0.5;

    size_t ws_bytes = 0;
    CALL(vegas_workspace_bytes(dim, nbins, iters, &ws_bytes));
    void *ws = NULL;
    cudaStream_t stream;
    CUDA(cudaMalloc(&ws, ws_bytes));
    CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));

    vegas_state *s = NULL;
    CALL(vegas_init_grid(&s, dim, nbins, seed, mode, VEGAS_GAUSS, params, 1 + dim, iters, ws,
                         ws_bytes, stream));
    for (int t = 0; t < k_adapt; ++t) {
        CALL(vegas_iterate(s, n_adapt, 1));
        CALL(vegas_refine(s, 1.5));
    }
    for (int t = 0; t < k_fixed; ++t) CALL(vegas_iterate(s, n_fixed, 0));

    double rows[6 * 64];
    int n_rows = 0;
    CALL(vegas_get_iterations(s, rows, iters < 64 ? iters : 64, &n_rows));
    for (int t = 0; t < n_rows; ++t) printf("%s%.17g", t ? " " : "", rows[6 * t + 4]);
    printf("\n");
    double mean = 0, sigma = 0, chi2 = 0;
    int n_iter = 0;
    CALL(vegas_result(s, k_adapt < iters ? k_adapt : 0, &mean, &sigma, &chi2, &n_iter));
    printf("%.17g %.17g %.17g %d\n", mean, sigma, chi2, n_iter);

    CALL(vegas_destroy(s));
    CUDA(cudaStreamDestroy(stream));
    CUDA(cudaFree(ws));
    return 0;
}
