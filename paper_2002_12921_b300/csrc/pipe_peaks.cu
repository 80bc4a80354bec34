// vegas_pipe_peak: the peak rate of each pipe the iterate kernels draw on,
// measured on the device in use, so that a kernel's rate of each operation can
// be stated as a fraction of what the hardware delivers for it.
//
// Each benchmark kernel runs, in every thread of a grid that fills every SM,
// eight independent dependency chains of one operation (the chains hide the
// operation's latency; the grid size, from the occupancy calculator, hides the
// rest).  Rate = threads x iterations x 8 / CUDA-event time of one launch after
// one warm-up launch.  Block 0 reads the SM cycle counter and the global timer
// at its start and end, which gives the SM clock during the launch.  The
// results feed a data-dependent store that never fires in practice, so no chain
// can be removed.
//
//   FFMA        fmaf(a, b, c) on floats
//   DFMA        fma on doubles
//   EX2         ex2.approx.ftz.f32 (the exponential's special-function step)
//   PRODUCT     a 32x32 -> 64-bit product as umulhi + low multiply, the form
//               Philox and the bin split use
//   IMAD        a 32-bit multiply-add (low word), x <- x x + K
//   LDS         32-bit shared-memory loads, conflict free (a pointer chase)
//   ATOMS_U32   32-bit integer atomic adds to shared memory, conflict free
//   ATOMS_F32   float atomic adds to shared memory (the histogram's operation)
#include <cstdint>

#include <cuda_runtime.h>

#include "vegas_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kLdsWords = 4096;                          // 16 KB pointer-chase table
constexpr int kAtomWords = kThreads / 32 * kChains * 32;  // 8 KB: one word per warp, chain, lane

struct PeakOut {
    unsigned long long sink;   // written only when a chain hits a value it never reaches
    unsigned long long clk0, clk1, ns0, ns1;
};

__device__ __forceinline__ unsigned long long global_ns_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mark(PeakOut* out, bool end) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long c = clock64(), t = global_ns_now();
        if (end) {
            out->clk1 = c;
            out->ns1 = t;
        } else {
            out->clk0 = c;
            out->ns0 = t;
        }
    }
}

// `never` is a kernel argument, so the compiler cannot prove the store dead
__device__ __forceinline__ void keep(PeakOut* out, uint32_t v, uint32_t never) {
    if (v == never) out->sink = v;
}

template <int OP>
__global__ void __launch_bounds__(kThreads) pipe_peak_kernel(uint32_t iters, uint32_t seed,
                                                             float fb, float fc, uint32_t never,
                                                             PeakOut* out) {
    mark(out, false);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t s = seed + blockIdx.x * kThreads + threadIdx.x;
    if constexpr (OP == VEGAS_PIPE_FFMA || OP == VEGAS_PIPE_EX2) {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = 0.25f + 0.5f * (float)((s + c) & 255u) / 256.0f;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if constexpr (OP == VEGAS_PIPE_FFMA) {
                    a[c] = fmaf(a[c], fb, fc);
                } else {  // x <- 2^-x stays in (0.5, 1)
                    asm volatile("{ .reg .f32 t; neg.f32 t, %1; ex2.approx.ftz.f32 %0, t; }"
                                 : "=f"(a[c]) : "f"(a[c]));
                }
            }
        }
        float t = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) t += a[c];
        keep(out, __float_as_uint(t), never);
    } else if constexpr (OP == VEGAS_PIPE_DFMA) {
        double a[kChains];
        const double b = fb, cc = fc;
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = 0.25 + 0.5 * (double)((s + c) & 255u) / 256.0;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, cc);
        }
        double t = 0.0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) t += a[c];
        keep(out, (uint32_t)__double2hiint(t) ^ (uint32_t)__double2loint(t), never);
    } else if constexpr (OP == VEGAS_PIPE_PRODUCT || OP == VEGAS_PIPE_IMAD) {
        constexpr uint32_t kM = 0xD2511F53u, kK = 0x9E3779B9u;
        uint32_t x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = s * (2u * c + 1u) + c;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if constexpr (OP == VEGAS_PIPE_PRODUCT)
                    x[c] = __umulhi(kM, x[c]) ^ (kM * x[c]);
                else  // nonlinear, so unrolled steps cannot be folded into one
                    x[c] = x[c] * x[c] + kK;
            }
        }
        uint32_t t = 0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) t ^= x[c];
        keep(out, t, never);
    } else if constexpr (OP == VEGAS_PIPE_LDS) {
        // table word p holds the shared address of word (p + 32) mod size: the
        // same bank, so a warp's 32 lanes (distinct banks) never conflict
        __shared__ uint32_t table[kLdsWords];
        const uint32_t base = (uint32_t)__cvta_generic_to_shared(table);
        for (int p = threadIdx.x; p < kLdsWords; p += kThreads)
            table[p] = base + 4u * (uint32_t)((p + 32) % kLdsWords);
        __syncthreads();
        uint32_t v[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c)  // chain c of a lane starts at lane + 512 c
            v[c] = base + 4u * (lane + 32u * (16u * c + (warp & 15u)));
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm volatile("ld.shared.u32 %0, [%0];" : "+r"(v[c]));
        }
        uint32_t t = 0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) t ^= v[c];
        keep(out, t, never);
    } else {  // ATOMS_U32, ATOMS_F32: one word per (warp, chain, lane)
        __shared__ uint32_t words[kAtomWords];
        for (int p = threadIdx.x; p < kAtomWords; p += kThreads) words[p] = 0u;
        __syncthreads();
        uint32_t* mine = words + warp * (kChains * 32) + lane;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if constexpr (OP == VEGAS_PIPE_ATOMS_U32)
                    atomicAdd(mine + 32 * c, 1u);
                else
                    atomicAdd(reinterpret_cast<float*>(mine + 32 * c), 1.0f);
            }
        }
        __syncthreads();
        keep(out, words[threadIdx.x], never);
    }
    __syncthreads();
    mark(out, true);
}

struct OpInfo {
    void (*kernel)(uint32_t, uint32_t, float, float, uint32_t, PeakOut*);
    uint32_t default_iters;  // about a millisecond per launch on a B300
};

OpInfo op_info(int op) {
    switch (op) {
        case VEGAS_PIPE_FFMA: return {pipe_peak_kernel<VEGAS_PIPE_FFMA>, 16384};
        case VEGAS_PIPE_DFMA: return {pipe_peak_kernel<VEGAS_PIPE_DFMA>, 256};
        case VEGAS_PIPE_EX2: return {pipe_peak_kernel<VEGAS_PIPE_EX2>, 2048};
        case VEGAS_PIPE_PRODUCT: return {pipe_peak_kernel<VEGAS_PIPE_PRODUCT>, 4096};
        case VEGAS_PIPE_IMAD: return {pipe_peak_kernel<VEGAS_PIPE_IMAD>, 8192};
        case VEGAS_PIPE_LDS: return {pipe_peak_kernel<VEGAS_PIPE_LDS>, 4096};
        case VEGAS_PIPE_ATOMS_U32: return {pipe_peak_kernel<VEGAS_PIPE_ATOMS_U32>, 2048};
        case VEGAS_PIPE_ATOMS_F32: return {pipe_peak_kernel<VEGAS_PIPE_ATOMS_F32>, 1024};
        default: return {nullptr, 0};
    }
}

}  // namespace

extern "C" int vegas_pipe_peak(int op, uint32_t iters, void* d_scratch, size_t scratch_bytes,
                               void* cuda_stream, double* out) {
    const OpInfo info = op_info(op);
    if (!info.kernel || !out || !d_scratch || scratch_bytes < VEGAS_PIPE_SCRATCH_BYTES ||
        reinterpret_cast<uintptr_t>(d_scratch) % 8 != 0 || iters > (1u << 24))
        return VEGAS_EINVAL;
    if (iters == 0) iters = info.default_iters;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, info.kernel, kThreads, 0) !=
            cudaSuccess || per_sm < 1)
        return VEGAS_ECUDA;
    const unsigned grid = (unsigned)(sms * per_sm);
    PeakOut* po = static_cast<PeakOut*>(d_scratch);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return VEGAS_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return VEGAS_ECUDA;
    }
    int rc = VEGAS_OK;
    float ms = 0.0f;
    // the sentinel is a value no chain is expected to end on (a false hit only
    // writes the unused sink word)
    const uint32_t never = 0x7f3a19c5u;
    info.kernel<<<grid, kThreads, 0, st>>>(iters, 1u, 0.999f, 0.001f, never, po);  // warm-up
    cudaEventRecord(e0, st);
    info.kernel<<<grid, kThreads, 0, st>>>(iters, 2u, 0.999f, 0.001f, never, po);
    cudaEventRecord(e1, st);
    PeakOut h{};
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaMemcpyAsync(&h, po, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || ms <= 0.0f)
        rc = VEGAS_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != VEGAS_OK) return rc;
    const double lane_ops = (double)grid * kThreads * (double)iters * kChains;
    out[0] = lane_ops / (ms * 1e-3);
    out[1] = h.ns1 > h.ns0 ? (double)(h.clk1 - h.clk0) / (double)(h.ns1 - h.ns0) * 1e3 : 0.0;
    out[2] = (double)sms;
    out[3] = (double)grid;
    return VEGAS_OK;
}
