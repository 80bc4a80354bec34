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

#include "vegas_internal.h"

namespace vegas {

namespace {

constexpr int kRefineThreads = 256;

// Sum over the block, result broadcast to every thread (fixed order).
__device__ double block_sum_all(double v, double* sbuf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sbuf[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sbuf[w];
        sbuf[32] = t;
    }
    __syncthreads();
    return sbuf[32];
}

__device__ double damp(double r, double alpha) {
    if (r <= 0.0) return 0.0;
    if (r == 1.0) return 1.0;
    return pow((r - 1.0) / log(r), alpha);
}

__global__ void __launch_bounds__(kRefineThreads) refine_kernel(const RefineArgs a) {
    extern __shared__ double sm[];
    __shared__ double sbuf[33];
    const int N = a.nbins;
    const int k = blockIdx.x;
    double* h = sm;            // N   histogram row
    double* m = h + N;         // N   smoothed, then damped weights
    double* C = m + N;         // N+1 cumulative weights
    double* eo = C + N + 1;    // N+1 old edges
    double* hist = a.hist + (size_t)k * N;
    double* edges = a.edges + (size_t)k * (N + 1);

    for (int j = threadIdx.x; j < N; j += blockDim.x) h[j] = hist[j];
    for (int l = threadIdx.x; l <= N; l += blockDim.x) eo[l] = edges[l];
    __syncthreads();

    double part = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) part += h[j];
    const double total = block_sum_all(part, sbuf);
    const bool refine = N >= 2 && total > 0.0 && total <= DBL_MAX;

    if (refine) {
        double ps = 0.0;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            double s;
            if (j == 0) s = (h[0] + h[1]) / 2.0;
            else if (j == N - 1) s = (h[N - 2] + h[N - 1]) / 2.0;
            else s = (h[j - 1] + h[j] + h[j + 1]) / 3.0;
            m[j] = s;
            ps += s;
        }
        const double ssum = block_sum_all(ps, sbuf);
        for (int j = threadIdx.x; j < N; j += blockDim.x) m[j] = damp(m[j] / ssum, a.alpha);
        __syncthreads();

        // inclusive scan of m into C[1..N] by warp 0, 32 bins at a time
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            double carry = 0.0;
            if (lane == 0) C[0] = 0.0;
            for (int base = 0; base < N; base += 32) {
                const int j = base + lane;
                double v = j < N ? m[j] : 0.0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double u = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += u;
                }
                if (j < N) C[j + 1] = carry + v;
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
        }
        __syncthreads();

        const double delta = C[N] / N;
        for (int l = 1 + threadIdx.x; l < N; l += blockDim.x) {
            const double target = l * delta;
            // smallest b in [0, N-1] with target <= C[b+1]
            int lo = 0, hi = N - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (target <= C[mid + 1]) hi = mid;
                else lo = mid + 1;
            }
            const int b = lo;
            edges[l] = eo[b] + (target - C[b]) / m[b] * (eo[b + 1] - eo[b]);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) hist[j] = 0.0;
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

}  // namespace

cudaError_t launch_refine(const RefineArgs& a, cudaStream_t stream) {
    const size_t smem = (size_t)(4 * a.nbins + 2) * sizeof(double);
    refine_kernel<<<a.dim, kRefineThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_init(double* edges, double* hist, double* log, unsigned* ctrl, int dim,
                        int nbins, int max_iters, cudaStream_t stream) {
    init_kernel<<<32, 256, 0, stream>>>(edges, hist, log, ctrl, dim, nbins,
                                       max_iters * kLogStride);
    return cudaGetLastError();
}

}  // namespace vegas
