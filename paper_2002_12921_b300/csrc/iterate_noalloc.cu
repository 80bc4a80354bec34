// vegas_iterate_noalloc: one Vegas iteration (plus the refinement when adapting)
// for callers that may not allocate device memory.
//
// Everything the iteration needs besides the caller's inputs and outputs -- the
// per-block partial sums, the last-block ticket and the (fJ)^2 histogram -- lives
// in one file-scope device array.  Host code may not use that array's name as a
// pointer (on the host it names a host-side stand-in, not device memory), so
// each call looks up the device's address of it with cudaGetSymbolAddress, with
// that device current, and passes it to the kernels.
#include <cfloat>
#include <cmath>
#include <cstring>
#include <mutex>

#include "iterate_kernel.cuh"

namespace vegas {
namespace {

constexpr int kNaMaxBlocks = VEGAS_NOALLOC_MAX_BLOCKS;
constexpr int kNaMaxDimBins = VEGAS_NOALLOC_MAX_DIM_X_BINS;
// scratch layout: partials | histogram | control words
constexpr size_t kNaPartials = 0;
constexpr size_t kNaHist = kNaPartials + (size_t)kNaMaxBlocks * kPartialStride * sizeof(double);
constexpr size_t kNaCtrl = kNaHist + (size_t)kNaMaxDimBins * sizeof(double);
constexpr size_t kNaBytes = kNaCtrl + kCtrlWords * sizeof(unsigned);
static_assert(kNaBytes == VEGAS_NOALLOC_SCRATCH_BYTES, "scratch size in vegas.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = kMaxDevices;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kNaMaxDevices] = {};

// The device address of the scratch on `device` (current).  A call made
// outside stream capture looks it up afresh, so that an address left stale by a
// context that was torn down and rebuilt (cudaDeviceReset) is never used; a
// call made while `stream` is capturing reuses the last lookup on that device.
cudaError_t scratch_address(int device, cudaStream_t stream, unsigned char** out) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

struct NoAllocArgs {
    const double* edges;
    double* hist;       // scratch
    double* partials;   // scratch
    unsigned* ticket;   // scratch
    double* out;        // caller: S1, S2, n, nonfinite, I, var
    unsigned long long n;
    unsigned iter;
    int nbins;
    int log2r;          // shared histogram copies (as in the iterate kernel)
    unsigned rk0[10], rk1[10];
    FnConsts fc;
    int rowoff[kMaxDim];  // k N: row offsets of the staged grid
};

// The iterate kernel with its scratch taken from the arguments above and its
// result written to the caller's six doubles (one launch per iteration, no
// pre-scale from a previous estimate).
template <typename R, int D, int FN, bool ADAPT>
__global__ void __launch_bounds__(256) noalloc_iterate_kernel(const NoAllocArgs a) {
    using P = Prec<R>;
    using Pair = typename P::Pair;
    using H = typename P::Hist;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sred[32];
    __shared__ unsigned sbad[32];
    __shared__ int s_last;

    const int N = a.nbins;
    const int logr = ADAPT ? a.log2r : 0;
    Pair* sgrid = reinterpret_cast<Pair*>(smem_raw);
    H* shist = reinterpret_cast<H*>(sgrid + D * N);
    stage_grid<R, D, ADAPT>(a.edges, N, logr, a.fc, sgrid, shist);
    R n4, nlast;
    jacobian_factors<R, D>(N, n4, nlast);
    __syncthreads();

    IterateSink<R, D, ADAPT> sink(shist, N, logr);
    sample_loop<R, D, Integrand<R, FN>>((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x,
                                        a.n, (unsigned long long)gridDim.x * blockDim.x, a.iter,
                                        0u, a.rk0, a.rk1, a.fc, N, a.rowoff,
                                        (R)(sizeof(R) == 4 ? a.fc.C32 : a.fc.C), n4, nlast, sgrid,
                                        sink);
    const Acc<R>& acc = sink.acc;
    const unsigned bad = sink.bad;

    const double b1 = acc.block1(reinterpret_cast<FloatFloat*>(sred));
    const double b2 = acc.block2(reinterpret_cast<FloatFloat*>(sred));
    const unsigned bb = block_sum(bad, sbad);
    if (ADAPT) {
        __syncthreads();
        flush_hist(shist, D * N, logr, 1.0, a.hist);
    }
    if (threadIdx.x == 0) {
        double* p = a.partials + (size_t)blockIdx.x * kPartialStride;
        p[0] = b1;
        p[1] = b2;
        p[2] = (double)bb;
        __threadfence();
        const unsigned ticket = atomicAdd(a.ticket, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double t1 = 0.0, t2 = 0.0, tb = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const double* p = a.partials + (size_t)b * kPartialStride;
        t1 += __ldcg(p + 0);
        t2 += __ldcg(p + 1);
        tb += __ldcg(p + 2);
    }
    t1 = block_sum(t1, sred);
    t2 = block_sum(t2, sred);
    tb = block_sum(tb, sred);
    if (threadIdx.x == 0) {
        const double n = (double)a.n;
        const double I = t1 / n;
        const double var = (t2 / n - I * I) / (n - 1.0);
        a.out[0] = t1;
        a.out[1] = t2;
        a.out[2] = n;
        a.out[3] = tb;
        a.out[4] = I;
        a.out[5] = var > 0.0 ? var : 0.0;
        *a.ticket = 0u;
    }
}

#define NA_ROW(R, D) \
    {(const void*)&noalloc_iterate_kernel<R, D, VEGAS_GAUSS, false>, \
     (const void*)&noalloc_iterate_kernel<R, D, VEGAS_GAUSS, true>}

const void* noalloc_kernel(int mode, int dim, bool adapt) {
    static const void* const f32[kMaxDim][2] = {
        NA_ROW(float, 1),  NA_ROW(float, 2),  NA_ROW(float, 3),  NA_ROW(float, 4),
        NA_ROW(float, 5),  NA_ROW(float, 6),  NA_ROW(float, 7),  NA_ROW(float, 8),
        NA_ROW(float, 9),  NA_ROW(float, 10), NA_ROW(float, 11), NA_ROW(float, 12),
        NA_ROW(float, 13), NA_ROW(float, 14), NA_ROW(float, 15), NA_ROW(float, 16),
        NA_ROW(float, 17), NA_ROW(float, 18), NA_ROW(float, 19), NA_ROW(float, 20)};
    static const void* const f64[kMaxDim][2] = {
        NA_ROW(double, 1),  NA_ROW(double, 2),  NA_ROW(double, 3),  NA_ROW(double, 4),
        NA_ROW(double, 5),  NA_ROW(double, 6),  NA_ROW(double, 7),  NA_ROW(double, 8),
        NA_ROW(double, 9),  NA_ROW(double, 10), NA_ROW(double, 11), NA_ROW(double, 12),
        NA_ROW(double, 13), NA_ROW(double, 14), NA_ROW(double, 15), NA_ROW(double, 16),
        NA_ROW(double, 17), NA_ROW(double, 18), NA_ROW(double, 19), NA_ROW(double, 20)};
    return (mode == VEGAS_FP32_EVAL ? f32 : f64)[dim - 1][adapt ? 1 : 0];
}

struct Guard {
    int prev = -1;
    bool ok = true;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~Guard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace vegas

extern "C" int vegas_iterate_noalloc(double* d_edges, int dim, int nbins, uint64_t seed,
                                     uint32_t iter, int mode, const double* params, int nparams,
                                     uint64_t n_samples, int adapt, double alpha,
                                     double* d_result, void* cuda_stream) {
    vegas::TraceRange trace_("vegas_iterate_noalloc");
    using namespace vegas;
    if (dim < 1 || dim > kMaxDim || nbins < 1 || nbins > kMaxBins) return VEGAS_EINVAL;
    if (dim * nbins > kNaMaxDimBins) return VEGAS_ENOSPACE;
    if (mode != VEGAS_FP64 && mode != VEGAS_FP32_EVAL) return VEGAS_EINVAL;
    if (!d_edges || !d_result || !params || nparams < 1 + dim) return VEGAS_EINVAL;
    if (n_samples < 2 || n_samples > (1ull << 40)) return VEGAS_EINVAL;
    if (adapt && !(alpha >= 0.0 && std::isfinite(alpha))) return VEGAS_EINVAL;
    for (int i = 0; i < 1 + dim; ++i)
        if (!std::isfinite(params[i])) return VEGAS_EINVAL;
    const double a_width = params[0];
    if (!(a_width > 0.0)) return VEGAS_EINVAL;

    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, d_edges) != cudaSuccess ||
        attr.type != cudaMemoryTypeDevice || attr.device < 0 || attr.device >= kNaMaxDevices) {
        cudaGetLastError();
        return VEGAS_EINVAL;
    }
    // the result is written by the kernel: device memory on the grid's device
    cudaPointerAttributes rattr;
    if (cudaPointerGetAttributes(&rattr, d_result) != cudaSuccess ||
        rattr.type != cudaMemoryTypeDevice || rattr.device != attr.device) {
        cudaGetLastError();
        return VEGAS_EINVAL;
    }
    Guard g(attr.device);
    if (!g.ok) return VEGAS_ECUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    unsigned char* scratch = nullptr;
    if (scratch_address(attr.device, stream, &scratch) != cudaSuccess) return VEGAS_ECUDA;

    // Gaussian constants (Eq. 1), as for the workspace path
    NoAllocArgs a;
    std::memset(&a, 0, sizeof(a));
    if (make_consts(VEGAS_GAUSS, dim, nbins, params, nparams, &a.fc) != VEGAS_OK)
        return VEGAS_EINVAL;
    philox_round_keys(seed, a.rk0, a.rk1);
    a.edges = d_edges;
    a.hist = reinterpret_cast<double*>(scratch + kNaHist);
    a.partials = reinterpret_cast<double*>(scratch + kNaPartials);
    a.ticket = reinterpret_cast<unsigned*>(scratch + kNaCtrl);
    a.out = d_result;
    a.n = n_samples;
    a.iter = iter;
    a.nbins = nbins;
    fill_row_offsets(nbins, a.rowoff);

    // what must start at zero: the ticket and, when adapting, the histogram
    if (cudaMemsetAsync(scratch + kNaCtrl, 0, kCtrlWords * sizeof(unsigned), stream) != cudaSuccess)
        return VEGAS_ECUDA;
    if (adapt && cudaMemsetAsync(scratch + kNaHist, 0, (size_t)dim * nbins * sizeof(double),
                                 stream) != cudaSuccess)
        return VEGAS_ECUDA;

    const bool ad = adapt != 0;
    const void* kern = noalloc_kernel(mode, dim, ad);
    a.log2r = ad ? hist_log2r(mode, dim, nbins) : 0;
    const size_t smem = iterate_smem_bytes(mode, dim, nbins, ad, a.log2r);
    int occ = 0, sms = 0;
    if (prepare_launch(attr.device, kern, 256, smem, &occ) != cudaSuccess || occ < 1 ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, attr.device) != cudaSuccess)
        return VEGAS_ECUDA;
    long long grid = (long long)((n_samples + 256 * 8 - 1) / (256 * 8));
    if (grid > (long long)sms * occ) grid = (long long)sms * occ;
    if (grid > kNaMaxBlocks) grid = kNaMaxBlocks;
    void* args[] = {&a};
    if (cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(256), args, smem, stream) != cudaSuccess)
        return VEGAS_ECUDA;
    if (ad) {
        RefineArgs r{};  // no staged pairs: this path stages in the iterate kernel
        r.edges = d_edges;
        r.hist = a.hist;
        r.dim = dim;
        r.nbins = nbins;
        r.alpha = alpha;
        if (launch_refine(r, stream) != cudaSuccess) return VEGAS_ECUDA;
    }
    return VEGAS_OK;
}
