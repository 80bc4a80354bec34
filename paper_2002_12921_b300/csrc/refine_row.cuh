// Grid refinement of one dimension (one row), shared by the refine kernels.
// (Lepage 1978 Sec. 3 with the smoothing of Lepage's 1980 report; see
// refine.cu for the rule.)  All threads of the block take part; `sm` holds
// 4 N + 2 doubles, `sbuf` 33.
#pragma once

#include <cfloat>
#include <cuda_runtime.h>

namespace vegas {

// Sum over the block, result broadcast to every thread (fixed order).
__device__ __forceinline__ double block_sum_all(double v, double* sbuf) {
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

// Threads per block for refining rows of N bins: one per bin, in whole warps,
// at most `max_threads` (the rows are short and every phase ends in a block
// barrier, so idle warps only add to each barrier's wait).
inline int refine_threads(int N, int max_threads) {
    const int t = (N + 31) / 32 * 32;
    return t < 32 ? 32 : (t > max_threads ? max_threads : t);
}

__device__ __forceinline__ double damp(double r, double alpha) {
    if (r <= 0.0) return 0.0;
    if (r == 1.0) return 1.0;
    const double x = (r - 1.0) / log(r);
    // the usual alpha = 3/2 as x sqrt(x): the same power to an ulp, without
    // pow's logarithm and exponential on the slow FP64 pipe
    return alpha == 1.5 ? x * sqrt(x) : pow(x, alpha);
}

// Refine one row in place: edges (N+1), hist (N, cleared on return).
__device__ __forceinline__ void refine_row(double* edges, double* hist, int N, double alpha,
                                           double* sm, double* sbuf) {
    double* h = sm;            // N   histogram row
    double* m = h + N;         // N   smoothed, then damped weights
    double* C = m + N;         // N+1 cumulative weights
    double* eo = C + N + 1;    // N+1 old edges
    for (int j = threadIdx.x; j < N; j += blockDim.x) h[j] = hist[j];
    for (int l = threadIdx.x; l <= N; l += blockDim.x) eo[l] = edges[l];
    __syncthreads();

    double part = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) part += h[j];
    const double total = block_sum_all(part, sbuf);
    const bool refine = N >= 2 && total > 0.0 && total <= DBL_MAX;

    if (refine) {
        // (multiplications by 1/3 and by 1/sum instead of divisions: the same
        // values to an ulp, with fewer instructions on the slow FP64 pipe)
        constexpr double kThird = 1.0 / 3.0;
        double ps = 0.0;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            double s;
            if (j == 0) s = (h[0] + h[1]) * 0.5;
            else if (j == N - 1) s = (h[N - 2] + h[N - 1]) * 0.5;
            else s = (h[j - 1] + h[j] + h[j + 1]) * kThird;
            m[j] = s;
            ps += s;
        }
        const double inv_ssum = 1.0 / block_sum_all(ps, sbuf);
        for (int j = threadIdx.x; j < N; j += blockDim.x) m[j] = damp(m[j] * inv_ssum, alpha);
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

}  // namespace vegas
