// Grid refinement and state initialisation kernels.
//
// Refinement (VegasFlow Sec. 2.2, the after-iteration step; the rule is
// Lepage 1978 Sec. 3 with the smoothing of Lepage's 1980 report), for one
// dimension with histogram h_j = sum over its samples of (fJ)^2 in bin j:
//   smoothing   s_0 = (h_0 + h_1)/2, s_j = (h_{j-1} + h_j + h_{j+1})/3,
//               s_{N-1} = (h_{N-2} + h_{N-1})/2;
//   damping     m_j = ((r_j - 1)/ln r_j)^alpha, r_j = s_j / sum s
//               (m = 0 at r = 0, m = 1 at r = 1);
//   re-partition: with C_0 = 0, C_{b+1} = C_b + m_b, new edge l (1..N-1) lies
//               in the old bin b with C_b < l sum(m)/N <= C_{b+1}, at
//               e_b + (l sum(m)/N - C_b)/m_b (e_{b+1} - e_b); e_0, e_N stay.
// A dimension whose histogram sums to zero or is not finite keeps its grid.
// One block per dimension, everything in double; the histogram is cleared.
#include <cfloat>
#include <cuda_runtime.h>

#include "refine_row.cuh"
#include "stage.cuh"
#include "vegas_internal.h"

namespace vegas {

namespace {

constexpr int kRefineThreads = 256;

__global__ void __launch_bounds__(kRefineThreads) refine_kernel(const RefineArgs a) {
    extern __shared__ double sm[];
    __shared__ double sbuf[33];
    const int N = a.nbins;
    const int k = blockIdx.x;
    double* e = a.edges + (size_t)k * (N + 1);
    refine_row(e, a.hist + (size_t)k * N, N, a.alpha, sm, sbuf);
    if (a.staged32) {  // the float path's pairs of the new grid
        __syncthreads();
        stage_row32(e, N, a.sc32[k], a.sh32[k], a.staged32 + (size_t)k * N);
    }
}

struct Stage32Args {
    const double* edges;
    float2* staged;
    int nbins;
    double sc[kMaxDim], sh[kMaxDim];
};

// The float path's staged pairs of the current grid, one block per dimension.
__global__ void stage32_kernel(const Stage32Args a) {
    const int k = blockIdx.x, N = a.nbins;
    stage_row32(a.edges + (size_t)k * (N + 1), N, a.sc[k], a.sh[k], a.staged + (size_t)k * N);
}

// Uniform grid e_l = l/N, cleared histogram, log and control words.
__global__ void init_kernel(double* edges, double* hist, double* log, unsigned* ctrl, int dim,
                            int nbins, int log_doubles) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    for (int i = tid; i < dim * (nbins + 1); i += nth) {
        const int l = i % (nbins + 1);
        edges[i] = (double)l / nbins;
    }
    for (int i = tid; i < dim * nbins; i += nth) hist[i] = 0.0;
    for (int i = tid; i < log_doubles; i += nth) log[i] = 0.0;
    for (int i = tid; i < kCtrlWords; i += nth) ctrl[i] = 0u;
}

// Log rows from summed shard totals: row r (kLogStride doubles apart) gets
// S1, S2, n, nonfinite, I, var from totals[3 r .. 3 r + 2] = {S1, S2,
// nonfinite}.
__global__ void shard_row_kernel(double* rows, const double* totals, int count,
                                 unsigned long long n_total) {
    const double n = (double)n_total;
    for (int r = threadIdx.x; r < count; r += blockDim.x) {
        double* row = rows + (size_t)r * kLogStride;
        const double S1 = totals[3 * r], S2 = totals[3 * r + 1];
        const double I = S1 / n;
        const double var = (S2 / n - I * I) / (n - 1.0);
        row[0] = S1;
        row[1] = S2;
        row[2] = n;
        row[3] = totals[3 * r + 2];
        row[4] = I;
        row[5] = var > 0.0 ? var : 0.0;
    }
}

// The grid digest of vegas_grid_digest: sum over the edges i of
// bits(e_i) K_i mod 2^64, K_i = splitmix64(i) | 1 (Vigna's SplitMix64 output
// for the index), and its complement.  Unsigned sums wrap, so the order of the
// additions does not matter: one block, a strided loop, a shuffle tree.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long i) {
    unsigned long long z = (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) grid_digest_kernel(const double* edges, int n,
                                                          unsigned long long* out) {
    __shared__ unsigned long long part[8];
    unsigned long long h = 0ull;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        h += (unsigned long long)__double_as_longlong(edges[i]) * (splitmix64((unsigned)i) | 1ull);
    for (int o = 16; o > 0; o >>= 1) h += __shfl_down_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = h;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        out[0] = t;
        out[1] = ~t;
    }
}

}  // namespace

cudaError_t launch_grid_digest(const double* edges, int n, unsigned long long* out,
                               cudaStream_t stream) {
    return launch_kernel(grid_digest_kernel, dim3(1), dim3(256), 0, stream, edges, n, out);
}

cudaError_t launch_shard_rows(double* rows, const double* totals, int count,
                              unsigned long long n_total, cudaStream_t stream) {
    const int threads = count < 256 ? 32 * ((count + 31) / 32) : 256;
    return launch_kernel(shard_row_kernel, dim3(1), dim3(threads), 0, stream, rows, totals,
                         count, n_total);
}

cudaError_t launch_refine(const RefineArgs& a, cudaStream_t stream) {
    const size_t smem = (size_t)(4 * a.nbins + 2) * sizeof(double);
    return launch_kernel(refine_kernel, dim3(a.dim), dim3(refine_threads(a.nbins, kRefineThreads)),
                         smem, stream, a);
}

cudaError_t launch_stage32(const double* edges, float2* staged, int dim, int nbins,
                           const FnConsts& fc, cudaStream_t stream) {
    Stage32Args a;
    a.edges = edges;
    a.staged = staged;
    a.nbins = nbins;
    for (int k = 0; k < kMaxDim; ++k) {
        a.sc[k] = fc.sc[1][k];
        a.sh[k] = fc.sh[1][k];
    }
    return launch_kernel(stage32_kernel, dim3(dim), dim3(128), 0, stream, a);
}

cudaError_t launch_init(double* edges, double* hist, double* log, unsigned* ctrl, int dim,
                        int nbins, int max_iters, cudaStream_t stream) {
    return launch_kernel(init_kernel, dim3(32), dim3(256), 0, stream, edges, hist, log, ctrl, dim,
                         nbins, max_iters * kLogStride);
}

}  // namespace vegas
