// The Philox words of a range of samples, written out (vegas_sample_words).
// Uses the iterate kernel's device Philox and counter layout: sample i of
// iteration t, call q, has counter (i low, i high, q | integral_id << 8, t);
// dimension k takes word k mod 4 of call k / 4.
#include <cuda_runtime.h>

#include "philox.cuh"
#include "vegas_internal.h"

namespace vegas {
namespace {

struct WordsArgs {
    unsigned long long i0, n;
    unsigned integral_id, iter;
    int dim;
    unsigned rk0[10], rk1[10];
    uint32_t* out;
};

__global__ void sample_words_kernel(const WordsArgs a) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long r = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         r < a.n; r += stride) {
        const unsigned long long i = a.i0 + r;
        for (int q = 0; 4 * q < a.dim; ++q) {
            uint32_t w0 = (uint32_t)i, w1 = (uint32_t)(i >> 32), w2 = (a.integral_id << 8) | q,
                     w3 = a.iter;
            philox4x32_10(w0, w1, w2, w3, a.rk0, a.rk1);
            const uint32_t w[4] = {w0, w1, w2, w3};
            for (int t = 0; t < 4 && 4 * q + t < a.dim; ++t)
                a.out[r * (unsigned long long)a.dim + 4 * q + t] = w[t];
        }
    }
}

}  // namespace
}  // namespace vegas

extern "C" int vegas_sample_words(uint64_t seed, uint32_t integral_id, uint32_t iter, uint64_t i0,
                                  uint64_t n, int dim, uint32_t* d_out, void* cuda_stream) {
    using namespace vegas;
    if (dim < 1 || dim > kMaxDim || (n > 0 && !d_out) || n > VEGAS_MAX_SAMPLE_INDEX)
        return VEGAS_EINVAL;
    if (n == 0) return VEGAS_OK;
    if (!device_memory_on(d_out, -1)) return VEGAS_EINVAL;
    WordsArgs a;
    a.i0 = i0;
    a.n = n;
    a.integral_id = integral_id;
    a.iter = iter;
    a.dim = dim;
    a.out = d_out;
    philox_round_keys(seed, a.rk0, a.rk1);
    unsigned long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    return launch_kernel(sample_words_kernel, dim3((unsigned)blocks), dim3(256), 0,
                         static_cast<cudaStream_t>(cuda_stream), a) == cudaSuccess
               ? VEGAS_OK
               : VEGAS_ECUDA;
}
