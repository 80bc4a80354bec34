// Philox4x32-10 words from cuRAND's device API, for checking the library's
// generator against a second implementation.  curand_init(seed, s, 4 i)
// starts a Philox4_32_10 state at counter (i lo, i hi, s lo, s hi) under key
// (seed lo, seed hi); curand4 then returns that counter's four words.  The
// library's counter of sample i is (i lo, i hi, q | integral_id << 8, iter), so
// s = iter << 32 | (q | integral_id << 8).
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void curand_words_kernel(uint64_t seed, uint64_t subsequence, uint64_t i0, uint64_t n,
                                    uint32_t* out) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    curandStatePhilox4_32_10_t state;
    curand_init(seed, subsequence, 4 * (i0 + t), &state);
    const uint4 r = curand4(&state);
    out[4 * t + 0] = r.x;
    out[4 * t + 1] = r.y;
    out[4 * t + 2] = r.z;
    out[4 * t + 3] = r.w;
}

// n x 4 words of counters (i0 + t, c2, c3) into d_out (device, n * 4 uint32).
extern "C" int curand_philox_words(uint64_t seed, uint32_t c2, uint32_t c3, uint64_t i0,
                                   uint64_t n, uint32_t* d_out, void* stream) {
    if (n == 0) return 0;
    if (!d_out || n > (1ull << 31)) return (int)cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    curand_words_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        seed, ((uint64_t)c3 << 32) | c2, i0, n, d_out);
    return (int)cudaGetLastError();
}
