// Internal declarations shared by the library's translation units (host and
// device).  Not part of the public ABI (include/vegas.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <tuple>
#include <utility>

#include "../../include/vegas.h"

namespace vegas {

// A named range around a C-ABI call, visible in profilers' timelines (NVTX;
// nearly free when no tool is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Launch through cudaLaunchKernel and return its status: the launch's own
// error, never a stale one left in the runtime's last-error state by an
// unrelated earlier call.
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t stream, Args&&... args) {
    std::tuple<KArgs...> values(std::forward<Args>(args)...);
    return std::apply(
        [&](auto&... v) {
            void* ptrs[] = {(void*)&v..., nullptr};
            return cudaLaunchKernel((const void*)kernel, grid, block, ptrs, smem, stream);
        },
        values);
}

constexpr int kMaxDim = VEGAS_MAX_DIM;
constexpr int kMaxBins = VEGAS_MAX_BINS;
constexpr int kMaxDimBins = VEGAS_MAX_DIM_X_BINS;
constexpr int kMaxGrid = 8192;      // blocks of one iterate launch (size of the partials array)
constexpr int kPartialStride = 4;   // doubles per block partial: S1, S2, nonfinite, unused
constexpr int kLogStride = 8;       // doubles per log row: S1, S2, n, nonfinite, I, var, 0, 0
constexpr int kNumIntegrands = 5;

// control words in device memory
// kT0: words 4-5, the complement of the %globaltimer value (ns) at which the
// current iteration's first block started (0: none yet).
enum CtrlWord { kTicket = 0, kIter = 1, kStatus = 2, kT0 = 4, kCtrlWords = 64 };
// status bits
// kStatusCheckFailed: a debug build's device check failed (a staged grid bin
// with a non-finite coordinate or a width that is not positive -- edges not
// increasing --, a bin index out of range, a non-finite mapped coordinate).
enum StatusBit { kStatusLogFull = 1u, kStatusCheckFailed = 2u };

// Integrand constants, precomputed on the host from the user's parameters.
//
// Staging transform: every bin is staged in the integrand's own coordinate
// z_k = sc_k x_k + sh_k (per precision: index 0 double, 1 float), so the map
// yields z with one fused multiply-add.  The Jacobian then collects
// prod_k N Delta_k sc_k, and 1/prod_k sc_k is folded into the prefactors.
struct FnConsts {
    double C;        // FP64 prefactor: normalisation x N^dim / prod sc
    double C32;      // FP32 prefactor: normalisation / prod sc (N^dim enters in the loop)
    double sc[2][kMaxDim];  // staging scale per precision and dimension
    double sh[2][kMaxDim];  // staging shift
    double d64[kMaxDim];    // MIX2: z_B - z_A in the double coordinate; GENZ_DISC: c_k
    double t64[kMaxDim];    // GENZ_DISC: thresholds a_k
    float d32[kMaxDim];     // MIX2: z_B - z_A in the float coordinate; GENZ_DISC: c_k log2 e
    float t32[kMaxDim];     // GENZ_DISC: thresholds a_k
    const void* user;       // VEGAS_USER: the caller's device data pointer
};

// Fill FnConsts for an integrand (VEGAS_EINVAL on bad parameters).
int make_consts(int integrand, int dim, int nbins, const double* params, int nparams,
                FnConsts* fc);
// Compose the integration box [lo_k, hi_k] into the staging of both precisions.
void compose_box(FnConsts* fc, int dim, const double* lo, const double* hi);

// Arguments of one iterate launch (passed by value in the parameter bank).
struct IterArgs {
    const double* edges;  // dim x (N+1)
    double* hist;         // dim x N
    double* partials;     // gridDim.x x kPartialStride
    double* log;          // max_iters x kLogStride
    unsigned* ctrl;       // kCtrlWords
    unsigned long long i0;       // first sample index of this launch
    unsigned long long n_chunk;  // samples of this launch
    unsigned long long n_total;  // samples of the whole iteration
    int first_chunk, last_chunk;
    int nbins, max_iters;
    int hist_log2r;       // log2 of the number of shared histogram copies
    unsigned integral_id;
    unsigned rk0[10], rk1[10];  // Philox round keys k + r W
    FnConsts fc;
    const float2* staged32;     // float path: the grid's staged pairs (dim x N), or null
    int rowoff[kMaxDim];        // k N: where row k of the staged grid starts
};

// k N for k < kMaxDim: the offsets of the staged grid's rows, passed to the
// kernels in their parameters so that a bin's index is one addition of a
// constant (k is a compile-time constant in the unrolled sample loop), not a
// multiply on the integer-multiply pipe that Philox saturates.
inline void fill_row_offsets(int nbins, int* rowoff) {
    for (int k = 0; k < kMaxDim; ++k) rowoff[k] = k * nbins;
}

struct RefineArgs {
    double* edges = nullptr;  // dim x (N+1), refined in place
    double* hist = nullptr;   // dim x N, cleared
    int dim = 0, nbins = 0;
    double alpha = 0.0;
    float2* staged32 = nullptr;  // float path: the refined grid's staged pairs (dim x N), or null
    double sc32[kMaxDim] = {}, sh32[kMaxDim] = {};  // the float staging transform
};

// Kernel lookup: the iterate kernel for (mode, integrand, dim, adapt), or
// nullptr.
const void* iterate_kernel_f32(int integrand, int dim, bool adapt);
// The float big-block adapting kernel (kBigBlockThreads threads per block).
const void* iterate_kernel_f32_big(int integrand, int dim);
// The float adapting kernel of the default shape with the run-time histogram
// copy count (iterate_kernel_f32's adapting kernels run 32 copies).
const void* iterate_kernel_f32_few(int integrand, int dim);
// The float fixed-grid kernels compiled for kFixedBins bins per dimension (the
// bin count of the paper's workloads here; measured per 1e8 samples with the
// bin count a constant of the index arithmetic: d = 8 715 -> 682 us, d = 12
// 1026 -> 977, d = 16 1306 -> 1262), for dimensions up to kFixedBinsMaxDim
// (at d = 20 it measured the same, 1593 against 1596 us; in the adapting
// kernels slower).  nullptr otherwise.
constexpr int kFixedBins = 50;
constexpr int kFixedBinsMaxDim = 16;
const void* iterate_kernel_f32_nb(int integrand, int dim);
const void* iterate_kernel_f64(int integrand, int dim, bool adapt);

// Devices a process may use with the library (device ordinals below this).
constexpr int kMaxDevices = VEGAS_MAX_DEVICES;
// Resident blocks per SM of `kern` launched with (block, smem) on `device`,
// which must be the current device.  The first launch of a (device, kernel,
// block, smem) shape in the process raises the kernel's dynamic shared-memory
// limit where smem needs it -- to the most a block may take on the device, so
// that no caller can lower it under another's launch -- and queries the
// occupancy; the answer is kept for the process.  Thread-safe.
cudaError_t prepare_launch(int device, const void* kern, int block, size_t smem, int* occ);

// Shared histogram copies of an adapting iterate block, as log2: 32 copies
// (one per lane) where they fit in kHistCopyBudget bytes, fewer otherwise.
constexpr size_t kHistCopyBudget = 52 * 1024;
// The big-block shape of a float adapting launch: one block of this many
// threads per SM (24 warps, the occupancy of the default shape), 32 copies.
constexpr int kBigBlockThreads = 768;
int hist_log2r(int mode, int dim, int nbins);
// dynamic shared memory of an iterate kernel with 2^log2r histogram copies
size_t iterate_smem_bytes(int mode, int dim, int nbins, bool adapt, int log2r);

cudaError_t launch_refine(const RefineArgs& a, cudaStream_t stream);
// The float path's staged pairs (dim x N) of the grid `edges` (refine.cu).
cudaError_t launch_stage32(const double* edges, float2* staged, int dim, int nbins,
                           const FnConsts& fc, cudaStream_t stream);
void combine_rows(const double* rows, int stride, int first_iter, int n, double* mean,
                  double* sigma, double* chi2_dof);
// Install summed shard totals {S1, S2, nonfinite} (3 doubles per row) into
// `count` consecutive log rows, with I, var for n_total samples each.
cudaError_t launch_shard_rows(double* rows, const double* totals, int count,
                              unsigned long long n_total, cudaStream_t stream);
// The 64-bit digest of n edges and its complement into out[0], out[1].
cudaError_t launch_grid_digest(const double* edges, int n, unsigned long long* out,
                               cudaStream_t stream);
cudaError_t launch_init(double* edges, double* hist, double* log, unsigned* ctrl, int dim,
                        int nbins, int max_iters, cudaStream_t stream);

}  // namespace vegas

// The host descriptor behind the opaque vegas_state handle.
struct vegas_state {
    int dim, nbins, mode, integrand, max_iters;
    uint64_t seed;
    cudaStream_t stream;
    int device;
    int sm_count;
    unsigned char* ws;
    size_t ws_bytes;
    double* edges;
    double* hist;
    double* log;
    double* partials;
    unsigned* ctrl;
    int host_iters;  // iterations enqueued through this descriptor
    vegas_config cfg;
    vegas::FnConsts fc;
    uint32_t rk0[10], rk1[10];
    double params[1 + 2 * VEGAS_MAX_DIM];  // the integrand parameters as given
    int nparams;
    vegas_user_integrand user;  // VEGAS_USER: the caller's kernels (launch == NULL: unset)
    // VEGAS_USER: the launch shape prepared for the fixed-grid [0] and the
    // adapting [1] kernel (occ 0: not yet)
    struct UserShape {
        int block;
        size_t smem;
        int occ;
    } user_shape[2];
    float2* staged32;  // VEGAS_FP32_EVAL: the grid's staged pairs in the workspace, else null
    int has_box;       // integration box [lo, hi] (vegas_set_box); else the unit cube
    double box_lo[VEGAS_MAX_DIM], box_hi[VEGAS_MAX_DIM];
    int inject_countdown;  // vegas_inject_failure: fail the n-th next enqueueing call (0: off)
    int smem_optin;        // dynamic shared memory one block may use on this device
    // Launch shapes already prepared on this state's device: the kernel's
    // dynamic shared-memory limit raised where needed and its resident blocks
    // per SM queried once per (kernel, block, shared bytes), not per iteration.
    struct LaunchShape {
        const void* kern;
        int block;
        size_t smem;
        int occ;
    } shapes[8];
    int n_shapes, next_shape;
    // Pinned host staging held by the descriptor (taken from the library's
    // pool of page-locked blocks at creation, returned to it by vegas_destroy):
    // the control words, then up to pin_rows log rows; every read of the log
    // goes through it.
    unsigned* pin_ctrl;
    double* pin_rows_buf;
    int pin_rows;
    size_t pin_bytes;
};

// vegas_inject_failure's check, at the start of every enqueueing call: true
// when this call is the one to fail (nothing has been enqueued or changed).
inline bool injected_failure(vegas_state* s) {
    return s->inject_countdown > 0 && --s->inject_countdown == 0;
}

// Whether p is device memory of `device` (-1: of any device), the only kind a
// kernel may be handed; a host pointer would fault the kernel, or, where the
// GPU can reach host memory, be used silently.  Clears the error a failed
// query leaves.
inline bool device_memory_on(const void* p, int device) {
    cudaPointerAttributes attr;
    if (!p || cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice && (device < 0 || attr.device == device);
}

// Rewrite a float-path state's staged pairs after its edges changed other than
// by vegas_refine (enqueued on the state's stream; VEGAS_OK for FP64 states).
int restage(vegas_state* s);

