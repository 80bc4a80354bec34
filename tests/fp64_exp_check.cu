// The library's table-driven double exponential and the CUDA library's exp on
// the same points, for the accuracy test.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../paper_2002_12921_b300/csrc/fp64_exp.cuh"

__global__ void fp64_exp_kernel(const double* x, double* y, double* ref, uint64_t n) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] = vegas::fp64_exp(x[i]);
    ref[i] = exp(x[i]);
}

// d_y[i] = fp64_exp(d_x[i]), d_ref[i] = exp(d_x[i]) for i < n (device buffers).
extern "C" int fp64_exp_eval(const double* d_x, double* d_y, double* d_ref, uint64_t n,
                             void* stream) {
    if (n == 0) return 0;
    if (!d_x || !d_y || !d_ref || n > (1ull << 31)) return (int)cudaErrorInvalidValue;
    fp64_exp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_x, d_y, d_ref, n);
    return (int)cudaGetLastError();
}
