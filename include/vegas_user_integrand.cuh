/* Integrands written by the caller in CUDA C++ and run inside the library's
 * fused Vegas iteration (VegasFlow Sec. 2.3: integrands in C++ or CUDA
 * linked into the integrator; Sec. 2.2 / Lepage 1978 Sec. 2: the sampling,
 * grid map and accumulation around them).
 *
 * A user integrand is a default-constructible type with a device call
 * operator over one point of [0,1]^D:
 *
 *     struct MyIntegrand {
 *         template <typename R, int D>
 *         __device__ R operator()(const R (&x)[D], const void *data) const;
 *     };
 *
 * R is float (VEGAS_FP32_EVAL) or double (VEGAS_FP64); x holds the point's
 * coordinates in registers; data is the device pointer given to
 * vegas_set_user_integrand (NULL if none).  The operator is inlined into the
 * sample loop: it runs once per sample, after the D coordinates are mapped,
 * and its value times the Jacobian enters the sums and (when adapting) the
 * per-dimension histograms exactly as a built-in integrand's does.  A value
 * that is not finite is counted and left out of the sums.
 *
 * In one .cu file of the caller's module (compiled with nvcc for sm_103a,
 * -std=c++17, position independent when it is a shared library):
 *
 *     #include "vegas_user_integrand.cuh"
 *     VEGAS_USER_INTEGRAND(my_integrand_d8, MyIntegrand, 8)
 *
 * defines  extern "C" const vegas_user_integrand *my_integrand_d8(void);
 * which instantiates the iterate kernel of dimension 8 for both precisions
 * and both adapt flags, and returns the descriptor to pass to
 * vegas_set_user_integrand for a state created with integrand VEGAS_USER.
 * The kernels are launched by code of the caller's module, so its CUDA
 * runtime (static or shared) needs no link to the library's.
 *
 * This header includes the library's kernel source and must be used with
 * the library built from the same tree (vegas_set_user_integrand rejects a
 * descriptor whose argument block differs in size). */
#pragma once

#include "vegas.h"

#include "../paper_2002_12921_b300/csrc/iterate_kernel.cuh"

namespace vegas {

// The integrand interface of the sample loop (begin / add / value) over a
// user functor U: the D mapped coordinates are kept in registers (every
// index below is a compile-time constant once the loop is unrolled) and U is
// evaluated on the whole point.
template <typename R, int D, typename U>
struct UserPoint {
    R x[D];
    __device__ __forceinline__ void begin() {}
    __device__ __forceinline__ void add(int k, R v, const FnConsts&) { x[k] = v; }
    __device__ __forceinline__ R value(const FnConsts& fc) const { return U{}(x, fc.user); }
};

template <typename U, int D>
const void* user_kernel(int mode, int adapt) {
    if (mode == VEGAS_FP32_EVAL)
        return adapt ? (const void*)&vegas_user_iterate_kernel<float, D, UserPoint<float, D, U>, true>
                     : (const void*)&vegas_user_iterate_kernel<float, D, UserPoint<float, D, U>, false>;
    if (mode == VEGAS_FP64)
        return adapt
                   ? (const void*)&vegas_user_iterate_kernel<double, D, UserPoint<double, D, U>, true>
                   : (const void*)&vegas_user_iterate_kernel<double, D, UserPoint<double, D, U>, false>;
    return nullptr;
}

template <typename U, int D>
int user_prepare(int mode, int adapt, int block, size_t smem, int* blocks) {
    const void* k = user_kernel<U, D>(mode, adapt);
    if (!k || !blocks) return (int)cudaErrorInvalidValue;
    // the static shared memory (~0.5 KB) counts against the 48 KB default too.
    // The limit goes to the most a block of this kernel may take on the
    // device, not to this launch's size, so that a state with fewer bins cannot
    // lower it under another state's launch of the same kernel.
    if (smem > 40 * 1024) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
        if (e != cudaSuccess) return (int)e;
        const size_t cap = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes
                                                               : 0;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(smem > cap ? smem : cap));
        if (e != cudaSuccess) return (int)e;
    }
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, block, smem);
}

template <typename U, int D>
int user_launch(int mode, int adapt, const void* args, unsigned grid, unsigned block, size_t smem,
                void* stream) {
    const void* k = user_kernel<U, D>(mode, adapt);
    if (!k || !args) return (int)cudaErrorInvalidValue;
    void* argv[] = {const_cast<void*>(args)};
    return (int)cudaLaunchKernel(k, dim3(grid), dim3(block), argv, smem,
                                 static_cast<cudaStream_t>(stream));
}

}  // namespace vegas

#define VEGAS_USER_INTEGRAND(NAME, FUNCTOR, DIM)                                             \
    static_assert((DIM) >= 1 && (DIM) <= VEGAS_MAX_DIM, "dimension out of range");          \
    extern "C" const vegas_user_integrand* NAME(void) {                                      \
        static const vegas_user_integrand desc = {(DIM), sizeof(vegas::IterArgs),           \
                                                  &vegas::user_prepare<FUNCTOR, (DIM)>,      \
                                                  &vegas::user_launch<FUNCTOR, (DIM)>};      \
        return &desc;                                                                        \
    }
