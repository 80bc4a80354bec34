// vegas_gauss_adjoint: the fixed-grid Vegas estimate of the Eq. 1 Gaussian
// integral and its gradient with respect to the integrand parameters
// (mu_1..mu_d, a), from samples regenerated from their counters.
//
// On a frozen grid the samples x_i (and their weights J_i) do not depend on
// the parameters, so the estimator I = (1/n) sum_i f(x_i) J_i has the exact
// derivative dI/dtheta = (1/n) sum_i J_i df/dtheta(x_i) (the reparameterised
// estimator).  For f = (a sqrt(pi))^-d exp(-sum_k (x_k - mu_k)^2 / a^2):
//   df/dmu_k = f 2 (x_k - mu_k) / a^2,
//   df/da    = (f / a) (2 sum_k (x_k - mu_k)^2 / a^2 - d).
// The kernel recomputes every sample from its Philox counter -- nothing per
// sample is stored -- and reduces the d+2 sums and their squares (for the
// Monte Carlo variance of each component) with the same block / last-block
// scheme as the iterate kernel.
#include <cfloat>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "iterate_kernel.cuh"

namespace vegas {
namespace {

// The Gaussian in its staged coordinate (z = c (x - mu)/a, c = 1 for double,
// sqrt(log2 e) for float), keeping every z_k for the gradient.
template <typename R, int D>
struct GaussCoords {
    R z[D];
    R s;
    __device__ __forceinline__ void begin() { s = R(0); }
    __device__ __forceinline__ void add(int k, R zk, const FnConsts&) {
        z[k] = zk;
        s = Prec<R>::fma(zk, zk, s);
    }
    __device__ __forceinline__ R value(const FnConsts&) const {
        if (sizeof(R) == 4) return ex2_approx(-(float)s);
        return fp64_exp(-(double)s);
    }
};

struct AdjointArgs {
    const double* edges;
    double* partials;  // workspace: gridDim.x x kStride
    unsigned* ctrl;    // workspace control words (ticket)
    double* out;       // caller: values[d+2], variances[d+2], nonfinite
    unsigned long long n;
    unsigned iter;
    int nbins;
    unsigned rk0[10], rk1[10];
    FnConsts fc;
    double two_over_c2;              // 2 / c^2, for g_a = fw (2 s / c^2 - d)
    double scale[kMaxDim + 2];       // per component: 1, 2/(a c) (x d), 1/a
    int rowoff[kMaxDim];             // k N: row offsets of the staged grid
};

// Sums of one component's values and squares.  Double: plain sums.  Float:
// plain float partial sums over a run of samples, each run's partials then
// added into Kahan-compensated sums (fold); a partial of kFold values carries
// a rounding of about kFold eps of its size, a few 1e-6 of the component's
// Monte Carlo error, and the run costs 2 float operations per sample instead
// of the compensated 8 -- with d + 2 components that is most of the float work.
constexpr int kFold = 64;
template <typename R>
struct AdjAcc;
template <>
struct AdjAcc<double> {
    double s1 = 0.0, s2 = 0.0;
    __device__ __forceinline__ void add(double v) {
        s1 += v;
        s2 = fma(v, v, s2);
    }
    __device__ __forceinline__ void fold() {}
    __device__ __forceinline__ double sum1() const { return s1; }
    __device__ __forceinline__ double sum2() const { return s2; }
};
template <>
struct AdjAcc<float> {
    float p1 = 0.f, p2 = 0.f;                  // the current run's plain sums
    float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;  // Kahan sums of the runs
    __device__ __forceinline__ void add(float v) {
        p1 += v;
        p2 = fmaf(v, v, p2);
    }
    __device__ __forceinline__ void fold() {
        const float y1 = p1 - c1;
        const float t1 = s1 + y1;
        c1 = (t1 - s1) - y1;
        s1 = t1;
        const float y2 = p2 - c2;
        const float t2 = s2 + y2;
        c2 = (t2 - s2) - y2;
        s2 = t2;
        p1 = p2 = 0.f;
    }
    __device__ __forceinline__ double sum1() const { return (double)s1 - (double)c1; }
    __device__ __forceinline__ double sum2() const { return (double)s2 - (double)c2; }
};

// Per component (I, d/dmu_k, d/da) the sums of the values and their squares;
// the count of non-finite weights.  The value-only pass keeps the iterate
// kernels' per-sample compensated sums (with one component the runs cost more
// than they save); finish() folds the last run.
template <typename R, int D, bool GRAD>
struct AdjointSink {
    static constexpr bool kNeedBins = false;
    static constexpr int NC = GRAD ? D + 2 : 1;
    static constexpr bool kRuns = GRAD && sizeof(R) == 4;
    typename std::conditional<kRuns, AdjAcc<R>, Acc<R>>::type acc[NC];
    unsigned bad = 0;
    int run = 0;
    R two_over_c2, dim;
    __device__ __forceinline__ AdjointSink(R t, R d) : two_over_c2(t), dim(d) {}
    template <typename F>
    __device__ __forceinline__ void operator()(R fw, const F& f, const uint32_t (&)[D]) {
        if (!Prec<R>::finite(fw)) {
            ++bad;
        } else {
            acc[0].add(fw);
            if (GRAD) {
#pragma unroll
                for (int k = 0; k < D; ++k) acc[1 + k].add(fw * f.z[k]);
                acc[D + 1].add(fw * Prec<R>::fma(f.s, two_over_c2, -dim));
            }
        }
        if (kRuns && ++run == kFold) finish();
    }
    __device__ __forceinline__ void finish() {
        if constexpr (kRuns) {
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c].fold();
            run = 0;
        }
    }
};

// NB > 0: the bin count compiled in (it must equal a.nbins), as for the
// float fixed-grid iterate kernels.
template <typename R, int D, bool GRAD, int NB = 0>
__global__ void __launch_bounds__(256) gauss_adjoint_kernel(const AdjointArgs a) {
    using P = Prec<R>;
    using Pair = typename P::Pair;
    constexpr int NC = GRAD ? D + 2 : 1;
    constexpr int kStride = 2 * NC + 1;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sred[32];
    __shared__ unsigned sbad[32];
    __shared__ int s_last;

    const int N = NB > 0 ? NB : a.nbins;
    Pair* sgrid = reinterpret_cast<Pair*>(smem_raw);
    stage_grid<R, D, false>(a.edges, N, 0, a.fc, sgrid, nullptr);
    R n4, nlast;
    jacobian_factors<R, D>(N, n4, nlast);
    __syncthreads();

    AdjointSink<R, D, GRAD> sink((R)a.two_over_c2, (R)D);
    sample_loop<R, D, GaussCoords<R, D>, AdjointSink<R, D, GRAD>, NB>(
        (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x, a.n,
        (unsigned long long)gridDim.x * blockDim.x, a.iter, 0u, a.rk0, a.rk1, a.fc, N, a.rowoff,
        (R)(sizeof(R) == 4 ? a.fc.C32 : a.fc.C), n4, nlast, sgrid, sink);
    sink.finish();

    double* part = a.partials + (size_t)blockIdx.x * kStride;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const double v1 = block_sum(sink.acc[c].sum1(), sred);
        const double v2 = block_sum(sink.acc[c].sum2(), sred);
        if (threadIdx.x == 0) {
            part[2 * c] = v1;
            part[2 * c + 1] = v2;
        }
    }
    const unsigned bb = block_sum(sink.bad, sbad);
    if (threadIdx.x == 0) {
        part[2 * NC] = (double)bb;
        __threadfence();
        const unsigned ticket = atomicAdd(&a.ctrl[kTicket], 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last block: reduce the partials in block order
    const double n = (double)a.n;
    for (int c = 0; c < kStride; ++c) {
        double t = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            t += __ldcg(a.partials + (size_t)b * kStride + c);
        t = block_sum(t, sred);
        if (threadIdx.x == 0) {
            if (c == 2 * NC) {
                a.out[2 * (D + 2)] = t;
            } else if ((c & 1) == 0) {
                a.out[c / 2] = a.scale[c / 2] * (t / n);
            } else {
                // the matching sum of values went to out[c/2] just before
                const int comp = c / 2;
                const double mean = a.out[comp] / a.scale[comp];
                const double var = (t / n - mean * mean) / (n - 1.0);
                a.out[D + 2 + comp] = a.scale[comp] * a.scale[comp] * (var > 0.0 ? var : 0.0);
            }
        }
    }
    if (threadIdx.x == 0) {
        if (!GRAD)
            for (int c = 1; c < D + 2; ++c) a.out[c] = a.out[D + 2 + c] = 0.0;
        a.ctrl[kTicket] = 0u;
    }
}

#define ADJ_ROW(R, D) \
    {(const void*)&gauss_adjoint_kernel<R, D, false>, (const void*)&gauss_adjoint_kernel<R, D, true>}

const void* adjoint_kernel(int mode, int dim, bool grad) {
    static const void* const f32[kMaxDim][2] = {
        ADJ_ROW(float, 1),  ADJ_ROW(float, 2),  ADJ_ROW(float, 3),  ADJ_ROW(float, 4),
        ADJ_ROW(float, 5),  ADJ_ROW(float, 6),  ADJ_ROW(float, 7),  ADJ_ROW(float, 8),
        ADJ_ROW(float, 9),  ADJ_ROW(float, 10), ADJ_ROW(float, 11), ADJ_ROW(float, 12),
        ADJ_ROW(float, 13), ADJ_ROW(float, 14), ADJ_ROW(float, 15), ADJ_ROW(float, 16),
        ADJ_ROW(float, 17), ADJ_ROW(float, 18), ADJ_ROW(float, 19), ADJ_ROW(float, 20)};
    static const void* const f64[kMaxDim][2] = {
        ADJ_ROW(double, 1),  ADJ_ROW(double, 2),  ADJ_ROW(double, 3),  ADJ_ROW(double, 4),
        ADJ_ROW(double, 5),  ADJ_ROW(double, 6),  ADJ_ROW(double, 7),  ADJ_ROW(double, 8),
        ADJ_ROW(double, 9),  ADJ_ROW(double, 10), ADJ_ROW(double, 11), ADJ_ROW(double, 12),
        ADJ_ROW(double, 13), ADJ_ROW(double, 14), ADJ_ROW(double, 15), ADJ_ROW(double, 16),
        ADJ_ROW(double, 17), ADJ_ROW(double, 18), ADJ_ROW(double, 19), ADJ_ROW(double, 20)};
    return (mode == VEGAS_FP32_EVAL ? f32 : f64)[dim - 1][grad ? 1 : 0];
}

// The float kernels compiled for kFixedBins bins, dimensions up to
// kFixedBinsMaxDim (nullptr otherwise): d=8 forward 0.714 -> 0.684 ms,
// backward 0.869 -> 0.828 ms per 1e8.
#define ADJ_ROW_NB(D)                                                          \
    {(const void*)&gauss_adjoint_kernel<float, D, false, kFixedBins>,          \
     (const void*)&gauss_adjoint_kernel<float, D, true, kFixedBins>}

const void* adjoint_kernel_nb(int dim, bool grad) {
    static const void* const f32[kFixedBinsMaxDim][2] = {
        ADJ_ROW_NB(1),  ADJ_ROW_NB(2),  ADJ_ROW_NB(3),  ADJ_ROW_NB(4),
        ADJ_ROW_NB(5),  ADJ_ROW_NB(6),  ADJ_ROW_NB(7),  ADJ_ROW_NB(8),
        ADJ_ROW_NB(9),  ADJ_ROW_NB(10), ADJ_ROW_NB(11), ADJ_ROW_NB(12),
        ADJ_ROW_NB(13), ADJ_ROW_NB(14), ADJ_ROW_NB(15), ADJ_ROW_NB(16)};
    if (dim < 1 || dim > kFixedBinsMaxDim) return nullptr;
    return f32[dim - 1][grad ? 1 : 0];
}

}  // namespace
}  // namespace vegas

extern "C" int vegas_gauss_adjoint(vegas_state* s, const double* params, int nparams,
                                   uint32_t iter, uint64_t n_samples, int grad,
                                   double* d_out) {
    vegas::TraceRange trace_("vegas_gauss_adjoint");
    using namespace vegas;
    if (!s || !params || nparams < 1 + s->dim || !device_memory_on(d_out, s->device))
        return VEGAS_EINVAL;
    if (n_samples < 2 || n_samples > (1ull << 40)) return VEGAS_EINVAL;
    AdjointArgs a;
    std::memset(&a, 0, sizeof(a));
    if (make_consts(VEGAS_GAUSS, s->dim, s->nbins, params, nparams, &a.fc) != VEGAS_OK)
        return VEGAS_EINVAL;
    // over a box the staged coordinate is still z = c (x - mu)/a with
    // x = lo + w u, so the derivative formulas in z hold unchanged
    if (s->has_box) compose_box(&a.fc, s->dim, s->box_lo, s->box_hi);
    const int dim = s->dim;
    const double width = params[0];
    // staged coordinate z = c (x - mu)/a: c = 1 (double), sqrt(log2 e) (float)
    const double c = s->mode == VEGAS_FP32_EVAL ? std::sqrt(1.4426950408889634) : 1.0;
    a.two_over_c2 = 2.0 / (c * c);
    a.scale[0] = 1.0;
    for (int k = 0; k < dim; ++k) a.scale[1 + k] = 2.0 / (width * c);
    a.scale[dim + 1] = 1.0 / width;
    a.edges = s->edges;
    a.partials = s->partials;
    a.ctrl = s->ctrl;
    a.out = d_out;
    a.n = n_samples;
    a.iter = iter;
    a.nbins = s->nbins;
    fill_row_offsets(s->nbins, a.rowoff);
    std::memcpy(a.rk0, s->rk0, sizeof(a.rk0));
    std::memcpy(a.rk1, s->rk1, sizeof(a.rk1));

    int prev_dev = -1;
    if (cudaGetDevice(&prev_dev) != cudaSuccess) return VEGAS_ECUDA;
    if (prev_dev != s->device && cudaSetDevice(s->device) != cudaSuccess) return VEGAS_ECUDA;
    int rc = VEGAS_OK;
    const bool g = grad != 0;
    const void* kern = adjoint_kernel(s->mode, dim, g);
    if (s->mode == VEGAS_FP32_EVAL && s->nbins == kFixedBins && adjoint_kernel_nb(dim, g))
        kern = adjoint_kernel_nb(dim, g);
    const size_t smem = iterate_smem_bytes(s->mode, dim, s->nbins, false, 0);
    int occ = 0;
    if (prepare_launch(s->device, kern, 256, smem, &occ) != cudaSuccess || occ < 1)
        rc = VEGAS_ECUDA;
    if (rc == VEGAS_OK) {
        // the block partials (2 (d+2) + 1 doubles each) must fit the workspace's area
        const int stride = 2 * (g ? dim + 2 : 1) + 1;
        long long grid = (long long)((n_samples + 256 * 8 - 1) / (256 * 8));
        long long cap = (long long)s->sm_count * occ;
        const long long fit = (long long)kMaxGrid * kPartialStride / stride;
        if (cap > fit) cap = fit;
        if (grid > cap) grid = cap;
        void* args[] = {&a};
        if (cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(256), args, smem, s->stream) !=
            cudaSuccess)
            rc = VEGAS_ECUDA;
    }
    if (prev_dev != s->device) cudaSetDevice(prev_dev);
    return rc;
}
