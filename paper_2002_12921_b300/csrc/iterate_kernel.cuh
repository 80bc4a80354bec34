// The fused Vegas iteration kernel: Philox4x32-10 -> grid map -> integrand ->
// per-thread sums -> block reduction -> privatised shared-memory histogram with
// one global flush per block -> last-block fixed-order tail reduction into the
// device iteration log.
//
// Method: VegasFlow Sec. 2.2 (the per-event step of the importance-sampling
// integrator) with the Vegas map and estimator of Lepage 1978 (cited in Sec. 1):
// for each sample, y in [0,1)^d picks bin j_k and a position inside it in every
// dimension, x_k = e_{k,j} + frac (e_{k,j+1} - e_{k,j}), the weight is
// J = prod_k N (e_{k,j+1} - e_{k,j}), and the iteration estimates I = <f J>,
// var = (<(fJ)^2> - I^2)/(n-1), while accumulating sum (fJ)^2 per (k, j_k) for
// the refinement.
//
// Two precisions share the structure:
//   double: map, integrand and all sums in double ("plain FP64");
//   float:  map and integrand in float; every thread keeps Kahan-compensated
//           float sums of f J and (f J)^2 and a float shared histogram, all
//           pre-scaled by 2^-h (h from the previous iteration's estimate) so
//           that no float sum overflows; everything above the thread is double.
#pragma once

#include <cfloat>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fp64_exp.cuh"
#include "philox.cuh"
#include "stage.cuh"
#include "vegas_internal.h"

// launch-shape tuning: minimum resident blocks the register allocation
// targets
#ifdef VEGAS_ITERATE_MIN_BLOCKS
#define VEGAS_ITERATE_BOUNDS __launch_bounds__(256, VEGAS_ITERATE_MIN_BLOCKS)
#else
#define VEGAS_ITERATE_BOUNDS __launch_bounds__(256)
#endif

namespace vegas {

// Samples per unrolled step of the sample loop.  Measured: two samples per
// step speed up the double kernels (d=8 Gaussian: fixed grid 8.49 -> 8.21 ms
// per 1e8, adapting 1.09 -> 1.06 ms per 1e7; 256-integral batch 61.5 -> 58.1
// ms) but slow the float ones (d=8 fixed grid 748 -> 773 us per 1e8; d=16
// mixture, adapting, 3.64e10 -> 3.29e10 samples/s; batch 7.95 -> 9.03 ms),
// whose integer-multiply pipe is already the busiest unit.
template <typename R>
constexpr int sample_unroll() {
    return sizeof(R) == 8 ? 2 : 1;
}

// 2^x with the hardware exponential (flush-to-zero for tiny results).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------------------
// Integrands, written in the staged coordinate z_k = sc_k x_k + sh_k (see
// FnConsts).  begin() resets the running state, add(k, z) folds in dimension k
// (a compile-time constant once the kernel's loops are unrolled, so the
// constants come straight from the parameter bank), value() returns f without
// its constant prefactor (which the kernel folds into the Jacobian).
// ------------------------------------------------------------------------
template <typename R, int FN>
struct Integrand;

// Eq. 1, float: z = kappa (x - mu), kappa^2 = log2(e)/a^2, f ~ 2^(-sum z^2).
template <>
struct Integrand<float, VEGAS_GAUSS> {
    float s;
    __device__ __forceinline__ void begin() { s = 0.f; }
    __device__ __forceinline__ void add(int, float z, const FnConsts&) { s = fmaf(z, z, s); }
    __device__ __forceinline__ float value(const FnConsts&) const { return ex2_approx(-s); }
};

// two-peak mixture, float: z_B = z_A + kappa (mu_A - mu_B).
template <>
struct Integrand<float, VEGAS_GAUSS_MIX2> {
    float sa, sb;
    __device__ __forceinline__ void begin() { sa = 0.f; sb = 0.f; }
    __device__ __forceinline__ void add(int k, float z, const FnConsts& c) {
        const float zb = z + c.d32[k];
        sa = fmaf(z, z, sa);
        sb = fmaf(zb, zb, sb);
    }
    __device__ __forceinline__ float value(const FnConsts&) const {
        return ex2_approx(-sa) + ex2_approx(-sb);
    }
};

template <>
struct Integrand<float, VEGAS_FLAT> {
    __device__ __forceinline__ void begin() {}
    __device__ __forceinline__ void add(int, float, const FnConsts&) {}
    __device__ __forceinline__ float value(const FnConsts&) const { return 1.f; }
};

// Eq. 2, float: z = x; zero unless every x_k > a_k, else 2^(sum c_k log2(e) x_k).
template <>
struct Integrand<float, VEGAS_GENZ_DISC> {
    float s;
    bool inside;
    __device__ __forceinline__ void begin() { s = 0.f; inside = true; }
    __device__ __forceinline__ void add(int k, float z, const FnConsts& c) {
        s = fmaf(z, c.d32[k], s);
        inside = inside && (z > c.t32[k]);
    }
    __device__ __forceinline__ float value(const FnConsts&) const {
        return inside ? ex2_approx(s) : 0.f;
    }
};

// Eq. 3, float: z = c (x - a), each factor c^2 / (1 + z^2); the c^2 and the
// normalisation sit in the prefactor.
template <>
struct Integrand<float, VEGAS_GENZ_PPEAK> {
    float p;
    __device__ __forceinline__ void begin() { p = 1.f; }
    __device__ __forceinline__ void add(int, float z, const FnConsts&) { p *= fmaf(z, z, 1.f); }
    __device__ __forceinline__ float value(const FnConsts&) const { return __fdividef(1.f, p); }
};

// Eq. 1, double: z = (x - mu)/a, f ~ exp(-sum z^2).
template <>
struct Integrand<double, VEGAS_GAUSS> {
    double s;
    __device__ __forceinline__ void begin() { s = 0.0; }
    __device__ __forceinline__ void add(int, double z, const FnConsts&) { s = fma(z, z, s); }
    __device__ __forceinline__ double value(const FnConsts&) const { return fp64_exp(-s); }
};

template <>
struct Integrand<double, VEGAS_GAUSS_MIX2> {
    double sa, sb;
    __device__ __forceinline__ void begin() { sa = 0.0; sb = 0.0; }
    __device__ __forceinline__ void add(int k, double z, const FnConsts& c) {
        const double zb = z + c.d64[k];
        sa = fma(z, z, sa);
        sb = fma(zb, zb, sb);
    }
    __device__ __forceinline__ double value(const FnConsts&) const {
        return fp64_exp(-sa) + fp64_exp(-sb);
    }
};

template <>
struct Integrand<double, VEGAS_FLAT> {
    __device__ __forceinline__ void begin() {}
    __device__ __forceinline__ void add(int, double, const FnConsts&) {}
    __device__ __forceinline__ double value(const FnConsts&) const { return 1.0; }
};

// Eq. 2, double: z = x.
template <>
struct Integrand<double, VEGAS_GENZ_DISC> {
    double s;
    bool inside;
    __device__ __forceinline__ void begin() { s = 0.0; inside = true; }
    __device__ __forceinline__ void add(int k, double z, const FnConsts& c) {
        s = fma(c.d64[k], z, s);
        inside = inside && (z > c.t64[k]);
    }
    __device__ __forceinline__ double value(const FnConsts&) const {
        return inside ? fp64_exp(s) : 0.0;
    }
};

// Eq. 3, double: z = c (x - a), f ~ 1 / prod_k (1 + z_k^2).
template <>
struct Integrand<double, VEGAS_GENZ_PPEAK> {
    double p;
    __device__ __forceinline__ void begin() { p = 1.0; }
    __device__ __forceinline__ void add(int, double z, const FnConsts&) { p *= fma(z, z, 1.0); }
    __device__ __forceinline__ double value(const FnConsts&) const { return 1.0 / p; }
};

// ------------------------------------------------------------------------
// Precision-specific pieces of the map.  unit(l) is the number in [1, 2) whose
// mantissa holds the position bits.  The staged pair of a bin is
// (sc e' + sh, sc Delta) with e' = e - (1 - u/2) Delta (u the unit's spacing),
// so that z = fma(unit, sc Delta, sc e' + sh) = sc (e + frac Delta) + sh with
// frac = unit - (1 - u/2) in (0, 1): for float frac = (floor(l / 2^9) + 1/2)
// 2^-23, for double frac = (l + 1/2) 2^-32.  One fused multiply-add gives the
// integrand's coordinate; the staged values are rounded once, which moves z by
// at most an ulp.
// ------------------------------------------------------------------------
template <typename R>
struct Prec;

template <>
struct Prec<float> {
    using Pair = float2;  // (shifted edge, width) of one bin, in shared memory
    using Hist = float;
    static __device__ __forceinline__ float unit(uint32_t l) {
        // (0x7F : l) >> 9 = 0x3F800000 | (l >> 9): one funnel shift
        return __uint_as_float(__funnelshift_r(l, 0x7Fu, 9));
    }
    static constexpr int kStage = 1;  // FnConsts staging index
    // (sc e' + sh, sc Delta) computed in double, rounded once
    static __device__ __forceinline__ Pair pair(double e0, double e1, double sc, double sh) {
        return stage_pair32(e0, e1, sc, sh);
    }
    static __device__ __forceinline__ bool finite(float v) { return fabsf(v) <= FLT_MAX; }
    static __device__ __forceinline__ float fma(float x, float y, float z) { return fmaf(x, y, z); }
};

template <>
struct Prec<double> {
    using Pair = double2;
    using Hist = double;
    static __device__ __forceinline__ double unit(uint32_t l) {
        // high word (0x3FF : l) >> 12 = 0x3FF00000 | (l >> 12), low word l << 20
        return __hiloint2double((int)__funnelshift_r(l, 0x3FFu, 12), (int)(l << 20));
    }
    static constexpr int kStage = 0;
    static __device__ __forceinline__ Pair pair(double e0, double e1, double sc, double sh) {
        const double w = e1 - e0;
        const double e = ::fma(-0x1.ffffffffp-1, w, e0);
        return make_double2(::fma(e, sc, sh), w * sc);
    }
    // exponent field not all ones, tested on the integer pipe (the same as
    // fabs(v) <= DBL_MAX, without an FP64 compare)
    static __device__ __forceinline__ bool finite(double v) {
        return ((unsigned)__double2hiint(v) & 0x7ff00000u) != 0x7ff00000u;
    }
    static __device__ __forceinline__ double fma(double x, double y, double z) {
        return ::fma(x, y, z);
    }
};

// Sum over the block in a fixed order (shuffle tree, then warp 0); the result
// is valid in thread 0.  sbuf holds 32 values.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sbuf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sbuf[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = ((int)threadIdx.x < nw) ? sbuf[threadIdx.x] : T(0);
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// A float-float value h + l (|l| <= ulp(h) / 2) and its sum: TwoSum of the
// high parts (exact), then the low parts, then renormalisation.  About 48
// significant bits, in FP32 instructions only.
struct FloatFloat {
    float h, l;
};

__device__ __forceinline__ FloatFloat ff_add(FloatFloat a, FloatFloat b) {
    const float s = a.h + b.h;
    const float v = s - a.h;
    const float e = (a.h - (s - v)) + (b.h - v);  // s + e == a.h + b.h exactly
    const float t = e + (a.l + b.l);
    const float h = s + t;
    return {h, t - (h - s)};
}

// Sum of per-thread float-float values over the block in a fixed order
// (shuffle tree, then warp 0), converted to double once, in thread 0: the
// float path's block reduction keeps FP64 instructions off every warp.
__device__ __forceinline__ double block_sum_ff(FloatFloat v, FloatFloat* sbuf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = ff_add(v, {__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)});
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sbuf[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (wid == 0) {
        v = lane < nw ? sbuf[lane] : FloatFloat{0.f, 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = ff_add(v, {__shfl_down_sync(0xffffffffu, v.h, o),
                           __shfl_down_sync(0xffffffffu, v.l, o)});
    }
    return (double)v.h + (double)v.l;
}

// Per-thread accumulators: compensated in float, plain in double.
template <typename R>
struct Acc;

template <>
struct Acc<float> {
    float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;
    // Kahan: c carries what the last addition rounded away (with its sign
    // flipped), and is taken off the next term.
    __device__ __forceinline__ void add(float v) {
        const float y1 = v - c1;
        const float t1 = s1 + y1;
        c1 = (t1 - s1) - y1;
        s1 = t1;
        const float y2 = fmaf(v, v, -c2);  // v^2 - c2 with one rounding
        const float t2 = s2 + y2;
        c2 = (t2 - s2) - y2;
        s2 = t2;
    }
    __device__ __forceinline__ double sum1() const { return (double)s1 - (double)c1; }
    __device__ __forceinline__ double sum2() const { return (double)s2 - (double)c2; }
    // the block totals of sum1 / sum2 (valid in thread 0)
    __device__ __forceinline__ double block1(FloatFloat* sbuf) const {
        return block_sum_ff(ff_add({s1, 0.f}, {-c1, 0.f}), sbuf);
    }
    __device__ __forceinline__ double block2(FloatFloat* sbuf) const {
        return block_sum_ff(ff_add({s2, 0.f}, {-c2, 0.f}), sbuf);
    }
};

template <>
struct Acc<double> {
    double s1 = 0.0, s2 = 0.0;
    __device__ __forceinline__ void add(double v) {
        s1 += v;
        s2 = fma(v, v, s2);
    }
    __device__ __forceinline__ double sum1() const { return s1; }
    __device__ __forceinline__ double sum2() const { return s2; }
    __device__ __forceinline__ double block1(FloatFloat* sbuf) const {
        return block_sum(s1, reinterpret_cast<double*>(sbuf));
    }
    __device__ __forceinline__ double block2(FloatFloat* sbuf) const {
        return block_sum(s2, reinterpret_cast<double*>(sbuf));
    }
};

// ------------------------------------------------------------------------
// Pieces shared by the iterate kernels.
//
// Shared memory of a block: the grid as D*N (shifted edge, width) pairs, then,
// when adapting, the histogram in 2^logr copies laid out [bin][copy]; lane L
// adds into copy L mod 2^logr, so lanes of one warp never update the same word
// (with 32 copies every lane also owns its bank).  Shared-memory float and
// double atomicAdd run as compare-and-swap loops, which then succeed at the
// first try.
// ------------------------------------------------------------------------
template <typename R, int D, bool ADAPT>
__device__ __forceinline__ void stage_grid(const double* __restrict__ edges, int N, int logr,
                                           const FnConsts& fc, typename Prec<R>::Pair* sgrid,
                                           typename Prec<R>::Hist* shist,
                                           const float2* __restrict__ staged32 = nullptr) {
    using P = Prec<R>;
    if (sizeof(R) == 4 && staged32 != nullptr) {
        // float path with the pairs already staged by the last grid change
        for (int idx = threadIdx.x; idx < D * N; idx += blockDim.x)
            reinterpret_cast<float2*>(sgrid)[idx] = staged32[idx];
    } else {
        for (int idx = threadIdx.x; idx < D * N; idx += blockDim.x) {
            const int k = idx / N, j = idx - k * N;
            const double* e = edges + (size_t)k * (N + 1) + j;
            sgrid[idx] = P::pair(e[0], e[1], fc.sc[P::kStage][k], fc.sh[P::kStage][k]);
        }
    }
    if (ADAPT)
        for (int idx = threadIdx.x; idx < (D * N) << logr; idx += blockDim.x)
            shist[idx] = typename P::Hist(0);
}

// The samples [first, end) with step `stride` of iteration `it`: Philox words
// (the first two rounds shared by a sample's calls), grid map, and the
// integrand F in its staged coordinate; each sample's weight f J, the
// integrand state and its bins go to sink(fw, f, bins), bins[k] = k N + j_k
// (the bin's index in the staged grid and in the histogram).  Returns whether the
// debug build's per-sample checks held (bin index < N, mapped coordinate
// finite); always true in the release build.
template <typename R, int D, typename F, typename Sink, int NB = 0>
__device__ __forceinline__ bool sample_loop(unsigned long long first, unsigned long long end,
                                            unsigned long long stride, unsigned it,
                                            uint32_t c2base, const unsigned (&rk0)[10],
                                            const unsigned (&rk1)[10], const FnConsts& fc,
                                            int N, const int (&rowoff)[kMaxDim], R jstart,
                                            R n4, R nlast,
                                            const typename Prec<R>::Pair* sgrid, Sink& sink) {
    using P = Prec<R>;
    using Pair = typename P::Pair;
    constexpr int DC = (D + 3) / 4;  // Philox calls per sample
    // Row k of the staged grid starts at k N.  Where the compiler can keep the
    // D products in registers (fixed-grid kernels up to d = 8) it does so, and
    // that measured fastest (d=8: 743 us per 1e8 against 772 us with the
    // offsets read from the parameters); with more dimensions, or the
    // adapting kernels' extra registers, it recomputes them on the
    // integer-multiply pipe, and the parameter offsets measured faster (d=16
    // fixed 1371 -> 1330 us, d=8 adapting 121.4 -> 119.2 us per 1e7).  With
    // the bin count compiled in (NB > 0) k N is an immediate at any D: d=12
    // fixed 1026 -> 977 us, d=16 1306 -> 1262 us per 1e8.
    constexpr bool kRowOff = (D > 8 && NB == 0) || Sink::kNeedBins;
    const uint32_t t_key = it ^ rk1[0];
    PhiloxCallConst pc[DC];
    bool checks_ok = true;
    // one sample, its index's low word i_lo (pc holds the high word's constants)
    auto one_sample = [&](uint32_t i_lo) {
        // rounds 0 and 1, shared by the calls: two wide multiplies per sample
        const uint32_t lo0 = kPhiloxM0 * i_lo;
        const uint32_t w2r0 = __umulhi(kPhiloxM0, i_lo) ^ t_key;
        const uint32_t hi1 = __umulhi(kPhiloxM1, w2r0);
        const uint32_t lo1 = kPhiloxM1 * w2r0;
        F f;
        f.begin();
        R J = jstart;
        uint32_t bins[D];
#pragma unroll
        for (int q = 0; q < DC; ++q) {
            uint32_t w0 = hi1 ^ pc[q].a, w1 = lo1, w2 = lo0 ^ pc[q].b, w3 = pc[q].c;
            philox_rounds<2, 10>(w0, w1, w2, w3, rk0, rk1);
            const uint32_t w[4] = {w0, w1, w2, w3};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int k = 4 * q + t;
                if (k < D) {
                    const uint32_t j = __umulhi(w[t], (uint32_t)N);
                    const uint32_t l = w[t] * (uint32_t)N;
                    const int gi = (kRowOff ? rowoff[k] : k * N) + (int)j;
                    const Pair g = sgrid[gi];
                    const R x = P::fma(P::unit(l), g.y, g.x);
#ifdef VEGAS_DEBUG_CHECKS
                    checks_ok &= j < (uint32_t)N && P::finite(x);
#endif
                    J *= g.y;
                    f.add(k, x, fc);
                    if (Sink::kNeedBins) bins[k] = (uint32_t)gi;
                }
            }
            if (sizeof(R) == 4) J *= (4 * q + 4 <= D) ? n4 : nlast;
        }
        sink(f.value(fc) * J, f, bins);
    };
    constexpr int kUnroll = sample_unroll<R>();
    // Two forms of the same loop over the thread's samples i = first, first +
    // stride, ... < end.  Segmented: in runs of one high word of i, counted in
    // 32 bits, the per-call constants fixed within a run -- fastest for the
    // fixed-grid kernels above d = 4 (d=8 744.6 -> 714.0 us per 1e8, d=16
    // 1333 -> 1304, d=20 1644 -> 1589).  Plain 64-bit loop with a check of the
    // high word: faster for d <= 4 (448.7 against 472.0 us) and not slower
    // for the adapting kernels.
    constexpr bool kSegmented = !Sink::kNeedBins && D > 4;
    if constexpr (kSegmented) {
        for (unsigned long long i = first; i < end;) {
            const uint32_t i_hi = (uint32_t)(i >> 32);
            // the next multiple of 2^32 (0 past the last one: the run goes to end)
            const unsigned long long next = ((unsigned long long)i_hi + 1ull) << 32;
            const unsigned long long seg_end = (next == 0ull || next > end) ? end : next;
            const uint32_t count = (uint32_t)((seg_end - i + stride - 1) / stride);
#pragma unroll
            for (int q = 0; q < DC; ++q)
                pc[q] = philox_call_const(c2base | (uint32_t)q, i_hi, rk0, rk1);
            uint32_t i_lo = (uint32_t)i;
#pragma unroll kUnroll
            for (uint32_t c = 0; c < count; ++c, i_lo += (uint32_t)stride) one_sample(i_lo);
            i += (unsigned long long)count * stride;
        }
    } else {
        uint32_t cur_hi = (uint32_t)(first >> 32);
#pragma unroll
        for (int q = 0; q < DC; ++q)
            pc[q] = philox_call_const(c2base | (uint32_t)q, cur_hi, rk0, rk1);
#pragma unroll kUnroll
        for (unsigned long long i = first; i < end; i += stride) {
            const uint32_t i_hi = (uint32_t)(i >> 32);
            if (i_hi != cur_hi) {  // crossing a multiple of 2^32: rare
                cur_hi = i_hi;
#pragma unroll
                for (int q = 0; q < DC; ++q)
                    pc[q] = philox_call_const(c2base | (uint32_t)q, i_hi, rk0, rk1);
            }
            one_sample((uint32_t)i);
        }
    }
    return checks_ok;
}

// Debug build: whether the grid the block runs on is well formed (per row of
// N + 1 edges: 0 and 1 at the ends, finite, strictly increasing).  It reads
// the edges themselves, so a grid corrupted in memory is seen whichever way
// the block staged it.
__device__ __forceinline__ bool edges_ok(const double* edges, int D, int N) {
    bool ok = true;
    for (int i = threadIdx.x; i < D * N; i += blockDim.x) {
        const int k = i / N, j = i - k * N;
        const double* e = edges + (size_t)k * (N + 1) + j;
        ok &= e[1] > e[0] && e[1] <= DBL_MAX;
        if (j == 0) ok &= e[0] == 0.0;
        if (j == N - 1) ok &= e[1] == 1.0;
    }
    return ok;
}

// Debug build: record a failed check in the state's status word (one atomic
// per block).  A barrier: every thread of the block calls it.
__device__ __forceinline__ void report_checks(bool ok, unsigned* ctrl) {
#ifdef VEGAS_DEBUG_CHECKS
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(&ctrl[kStatus], kStatusCheckFailed);
#else
    (void)ok;
    (void)ctrl;
#endif
}

// The iterate kernels' sink: per-thread sums of f J and (f J)^2, the count of
// non-finite weights, and (ADAPT) the shared histogram.
// The bit pattern of a histogram value, for compare-and-swap.
template <typename H>
struct HistBits;
template <>
struct HistBits<float> {
    using type = unsigned;
    static __device__ __forceinline__ unsigned bits(float v) { return __float_as_uint(v); }
};
template <>
struct HistBits<double> {
    using type = unsigned long long;
    static __device__ __forceinline__ unsigned long long bits(double v) {
        return (unsigned long long)__double_as_longlong(v);
    }
};

// LOGR >= 0: 2^LOGR copies known at compile time (the address of a bin's copy
// is then one shift-and-add of the bin index); -1: the run-time count lr.
template <typename R, int D, bool ADAPT, int LOGR = -1>
struct IterateSink {
    static constexpr bool kNeedBins = ADAPT;
    using H = typename Prec<R>::Hist;
    Acc<R> acc;
    unsigned bad = 0;
    H* hlane;  // this lane's copy: the histogram's base plus the lane's copy index
    int logr;
    uint32_t hbase;  // the lane's copy as a shared-memory address
    __device__ __forceinline__ IterateSink(H* h, int, int lr)
        : hlane(h + (threadIdx.x & ((1 << (LOGR >= 0 ? LOGR : lr)) - 1))),
          logr(LOGR >= 0 ? LOGR : lr) {
        hbase = (uint32_t)__cvta_generic_to_shared(hlane);
    }
    // the word of bin index i (= k N + j) in this lane's copy
    __device__ __forceinline__ H* at(uint32_t i) const {
        return hlane + ((int)i << (LOGR >= 0 ? LOGR : logr));
    }
    template <typename F>
    __device__ __forceinline__ void operator()(R fw, const F&, const uint32_t (&bins)[D]) {
        if (Prec<R>::finite(fw)) {
            acc.add(fw);
            if (ADAPT) {
                const R fw2 = fw * fw;
                if constexpr (sizeof(H) == 4) {
                    // The float shared-memory atomic add is a compare-and-swap
                    // loop on this GPU, and D of them in a row are D dependent
                    // round trips.  Groups of 4 dimensions instead: 4 loads, then
                    // 4 compare-and-swaps issued back to back, then a plain
                    // atomic add for any that lost a race with another warp
                    // (lanes own their copies, so within a warp none can).  One
                    // round trip per group: d=16 adapting iterations 6-9%
                    // faster, d=8 1%; a won swap stores old + v rounded to
                    // nearest, as the atomic add does.  (The double histograms
                    // keep the plain atomic add: the FP64 kernels are bound by
                    // the FP64 pipe, and grouping measured no faster there.)
                    // The loads and swaps address the lane's copy by its 32-bit
                    // shared-memory address (one shift-and-add per add): d=16
                    // adapting 199.5 -> 193.7 us per 1e7, the 256-integral
                    // batch's 8 iterations 6.04 -> 5.86 ms, d=8 unchanged.
                    using B = typename HistBits<H>::type;
                    const int sh = (LOGR >= 0 ? LOGR : logr) + 2;  // bytes per bin: 4 << logr
                    // one group of up to 8 dimensions where d <= 8 (d=8 116.6 ->
                    // 113.6 us per 1e7), groups of 4 above (groups of 8 there:
                    // d=16 193.7 -> 196.0, the batch's 8 iterations 5.86 ->
                    // 6.10 ms)
                    constexpr int G = D <= 8 ? 8 : 4;
#pragma unroll
                    for (int k0 = 0; k0 < D; k0 += G) {
                        uint32_t sa[G];
                        H old[G];
#pragma unroll
                        for (int g = 0; g < G; ++g)
                            if (k0 + g < D) {
                                sa[g] = hbase + (bins[k0 + g] << sh);
                                asm volatile("ld.shared.f32 %0, [%1];" : "=f"(old[g]) : "r"(sa[g]));
                            }
                        B got[G];
#pragma unroll
                        for (int g = 0; g < G; ++g)
                            if (k0 + g < D)
                                asm volatile("atom.shared.cas.b32 %0, [%1], %2, %3;"
                                             : "=r"(got[g])
                                             : "r"(sa[g]), "r"(HistBits<H>::bits(old[g])),
                                               "r"(HistBits<H>::bits(old[g] + (H)fw2))
                                             : "memory");
                        // one test for the group (any swap that lost a race),
                        // then the per-add tests only when one did: d=8
                        // adapting 119.5 -> 116.2 us per 1e7, d=20 238.6 ->
                        // 232.3 (groups of 8 this way: 119.7, 247.1)
                        B miss = 0;
#pragma unroll
                        for (int g = 0; g < G; ++g)
                            if (k0 + g < D) miss |= got[g] ^ HistBits<H>::bits(old[g]);
                        if (miss != 0) {
#pragma unroll
                            for (int g = 0; g < G; ++g)
                                if (k0 + g < D && got[g] != HistBits<H>::bits(old[g]))
                                    atomicAdd(at(bins[k0 + g]), (H)fw2);
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < D; ++k) atomicAdd(at(bins[k]), (H)fw2);
                }
            }
        } else {
            ++bad;
        }
    }
};

// Add the block's histogram (its copies summed, times scale) into the global
// one: one atomic per non-empty bin.  A thread sums one bin's R copies in the
// histogram's own type, starting at copy (bin mod R) so that the lanes of a
// warp read distinct banks; only the bin's total passes through double (on
// this GPU an FP64 warp instruction occupies the FP64 pipe ~60 cycles, so the
// flush keeps them to one conversion and one multiply per 32 bins).
template <typename H>
__device__ __forceinline__ void flush_hist(const H* shist, int nbins_total, int logr,
                                           double scale, double* hist) {
    const int m = (1 << logr) - 1;
    for (int b = threadIdx.x; b < nbins_total; b += blockDim.x) {
        const H* row = shist + (b << logr);
        H v = row[b & m];
        for (int c = 1; c <= m; ++c) v += row[(b + c) & m];
        if (v != (H)0) atomicAdd(&hist[b], (double)v * scale);
    }
}

// Jacobian start value and the float path's N^4 / N^(D mod 4) factors.
template <typename R, int D>
__device__ __forceinline__ void jacobian_factors(int N, R& n4, R& nlast) {
    n4 = (R)((double)N * N * N * N);
    double nrem = 1.0;
    for (int r = 0; r < D % 4; ++r) nrem *= N;
    nlast = (R)nrem;
}

// The GPU's global nanosecond timer.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------------
// The kernel body.  R = float or double, D = dimension, F = integrand type,
// ADAPT = accumulate the refinement histogram.
// ------------------------------------------------------------------------
// NB > 0: the bin count as a compile-time constant (it must equal a.nbins).
template <typename R, int D, typename F, bool ADAPT, int LOGR = -1, int NB = 0>
__device__ __forceinline__ void iterate_body(const IterArgs& a) {
    using P = Prec<R>;
    using Pair = typename P::Pair;
    using H = typename P::Hist;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sred[32];
    __shared__ unsigned sbad[32];
    __shared__ int s_last;

    const int N = NB > 0 ? NB : a.nbins;
    const int logr = ADAPT ? (LOGR >= 0 ? LOGR : a.hist_log2r) : 0;
    Pair* sgrid = reinterpret_cast<Pair*>(smem_raw);
    H* shist = reinterpret_cast<H*>(sgrid + D * N);

    const unsigned it = a.ctrl[kIter];
    if (it >= (unsigned)a.max_iters) {  // log full: the host refuses this too
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctrl[kStatus], kStatusLogFull);
        return;
    }
    // this block's start time, published after the samples (below)
    __shared__ unsigned long long s_start;
    if (threadIdx.x == 0) s_start = global_ns();
    stage_grid<R, D, ADAPT>(a.edges, N, logr, a.fc, sgrid, shist, a.staged32);

    // Pre-scale of the float path: f J is carried as f J 2^-h with 2^h near the
    // previous iteration's estimate; the prefactor enters the Jacobian's start.
    int h = 0;
    double j0;
    if (sizeof(R) == 4) {
        if (it > 0) {
            const double prev = a.log[(size_t)(it - 1) * kLogStride + 4];
            if (prev > 0.0 && prev <= DBL_MAX) h = max(-120, min(120, ilogb(prev)));
        }
        j0 = ldexp(a.fc.C32, -h);
    } else {
        j0 = a.fc.C;
    }
    R n4, nlast;
    jacobian_factors<R, D>(N, n4, nlast);
    __syncthreads();

    IterateSink<R, D, ADAPT, ADAPT ? LOGR : -1> sink(shist, N, logr);
    bool checks_ok = sample_loop<R, D, F, decltype(sink), NB>(
        a.i0 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x, a.i0 + a.n_chunk,
        (unsigned long long)gridDim.x * blockDim.x, it, a.integral_id << 8, a.rk0, a.rk1, a.fc,
        N, a.rowoff, (R)j0, n4, nlast, sgrid, sink);
#ifdef VEGAS_DEBUG_CHECKS
    checks_ok &= edges_ok(a.edges, D, N);
#endif
    report_checks(checks_ok, a.ctrl);
    const Acc<R>& acc = sink.acc;
    const unsigned bad = sink.bad;

    // Block reduction of the sums (fixed order), scaled back by 2^h / 2^2h.
    const double sc1 = ldexp(1.0, h), sc2 = ldexp(1.0, 2 * h);
    const double b1 = acc.block1(reinterpret_cast<FloatFloat*>(sred));
    const double b2 = acc.block2(reinterpret_cast<FloatFloat*>(sred));
    const unsigned bb = block_sum(bad, sbad);
    if (ADAPT) {
        __syncthreads();
        flush_hist(shist, D * N, logr, sc2, a.hist);
    }

    // Publish the block partial; the last block to finish reduces them all in
    // block order and appends the iteration to the log.
    // the iteration's start: the earliest block start of its first launch, kept
    // as a maximum of complements so that 0 means "not started"
    unsigned long long* t0c = reinterpret_cast<unsigned long long*>(a.ctrl + kT0);
    if (threadIdx.x == 0) {
        if (a.first_chunk) atomicMax(t0c, ~s_start);
        double* p = a.partials + (size_t)blockIdx.x * kPartialStride;
        p[0] = b1 * sc1;
        p[1] = b2 * sc2;
        p[2] = (double)bb;
        __threadfence();
        const unsigned ticket = atomicAdd(&a.ctrl[kTicket], 1u);
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
        double* L = a.log + (size_t)it * kLogStride;
        if (a.first_chunk) {
            L[0] = t1; L[1] = t2; L[2] = (double)a.n_chunk; L[3] = tb;
        } else {
            L[0] += t1; L[1] += t2; L[2] += (double)a.n_chunk; L[3] += tb;
        }
        if (a.last_chunk) {
            const double n = (double)a.n_total;
            const double I = L[0] / n;
            const double var = (L[1] / n - I * I) / (n - 1.0);
            L[4] = I;
            L[5] = var > 0.0 ? var : 0.0;
            // device time of the iteration: first block start to this point
            const unsigned long long c = *reinterpret_cast<volatile unsigned long long*>(t0c);
            L[6] = c ? (double)(global_ns() - ~c) : 0.0;
            L[7] = 0.0;
            *t0c = 0ull;
            a.ctrl[kIter] = it + 1;
        }
        a.ctrl[kTicket] = 0u;
    }
}

// The built-in integrands' kernel.  BIG: the instantiation for one block of
// up to kBigBlockThreads per SM (float adapting iterations whose 32
// lane-owned histogram copies fit that block's shared memory but not the
// default budget); its own launch bound leaves the default kernels' register
// allocation as it is.  LOGR: the histogram copies as a compile-time 2^LOGR
// (the float adapting kernels, whose launches use 32 copies but where they
// fit neither shape), -1 for the count in the arguments.
template <typename R, int D, int FN, bool ADAPT, bool BIG = false, int LOGR = -1, int NB = 0>
__global__ void __launch_bounds__(BIG ? kBigBlockThreads : 256)
    vegas_iterate_kernel(const IterArgs a) {
    iterate_body<R, D, Integrand<R, FN>, ADAPT, LOGR, NB>(a);
}

// the copies of the default table's adapting kernel: 32 for float, the
// run-time count for double
template <typename R>
constexpr int table_adapt_logr() {
    return sizeof(R) == 4 ? 5 : -1;
}

// The same kernel for an integrand type F supplied by the caller's own
// translation unit (include/vegas_user_integrand.cuh): F provides begin(),
// add(k, x, fc) and value(fc) in the plain coordinate x (the state must use
// VEGAS_USER, whose staging is the identity and whose prefactor is 1).
template <typename R, int D, typename F, bool ADAPT>
__global__ void VEGAS_ITERATE_BOUNDS vegas_user_iterate_kernel(const IterArgs a) {
    iterate_body<R, D, F, ADAPT>(a);
}

}  // namespace vegas

// Kernel table of one (precision, integrand): index [dim - 1][adapt].  The
// float adapting kernels of this table run 32 histogram copies.
#define VEGAS_KERNEL_ROW(R, FN, D) \
    {(const void*)&vegas::vegas_iterate_kernel<R, D, FN, false>, \
     (const void*)&vegas::vegas_iterate_kernel<R, D, FN, true, false, \
                                               vegas::table_adapt_logr<R>()>}

// The big-block adapting kernels of one float integrand: index [dim - 1].
#define VEGAS_KERNEL_TABLE_BIG(name, FN)                                                     \
    namespace vegas {                                                                         \
    const void* name(int dim) {                                                               \
        static const void* const table[kMaxDim] = {                                           \
            VEGAS_BIG(FN, 1),  VEGAS_BIG(FN, 2),  VEGAS_BIG(FN, 3),  VEGAS_BIG(FN, 4),          \
            VEGAS_BIG(FN, 5),  VEGAS_BIG(FN, 6),  VEGAS_BIG(FN, 7),  VEGAS_BIG(FN, 8),          \
            VEGAS_BIG(FN, 9),  VEGAS_BIG(FN, 10), VEGAS_BIG(FN, 11), VEGAS_BIG(FN, 12),         \
            VEGAS_BIG(FN, 13), VEGAS_BIG(FN, 14), VEGAS_BIG(FN, 15), VEGAS_BIG(FN, 16),         \
            VEGAS_BIG(FN, 17), VEGAS_BIG(FN, 18), VEGAS_BIG(FN, 19), VEGAS_BIG(FN, 20)};        \
        if (dim < 1 || dim > kMaxDim) return nullptr;                                         \
        return table[dim - 1];                                                                \
    }                                                                                         \
    }
#define VEGAS_BIG(FN, D) (const void*)&vegas::vegas_iterate_kernel<float, D, FN, true, true, 5>

// The float adapting kernels of one integrand with the run-time copy count
// (launches whose 32 copies fit neither shape): index [dim - 1].
#define VEGAS_KERNEL_TABLE_FEW(name, FN)                                                     \
    namespace vegas {                                                                         \
    const void* name(int dim) {                                                               \
        static const void* const table[kMaxDim] = {                                           \
            VEGAS_FEW(FN, 1),  VEGAS_FEW(FN, 2),  VEGAS_FEW(FN, 3),  VEGAS_FEW(FN, 4),          \
            VEGAS_FEW(FN, 5),  VEGAS_FEW(FN, 6),  VEGAS_FEW(FN, 7),  VEGAS_FEW(FN, 8),          \
            VEGAS_FEW(FN, 9),  VEGAS_FEW(FN, 10), VEGAS_FEW(FN, 11), VEGAS_FEW(FN, 12),         \
            VEGAS_FEW(FN, 13), VEGAS_FEW(FN, 14), VEGAS_FEW(FN, 15), VEGAS_FEW(FN, 16),         \
            VEGAS_FEW(FN, 17), VEGAS_FEW(FN, 18), VEGAS_FEW(FN, 19), VEGAS_FEW(FN, 20)};        \
        if (dim < 1 || dim > kMaxDim) return nullptr;                                         \
        return table[dim - 1];                                                                \
    }                                                                                         \
    }
#define VEGAS_FEW(FN, D) (const void*)&vegas::vegas_iterate_kernel<float, D, FN, true, false, -1>

// The float fixed-grid kernels of one integrand for kFixedBins bins per
// dimension, dimensions 1..kFixedBinsMaxDim: index [dim - 1].
#define VEGAS_KERNEL_TABLE_NB(name, FN)                                                      \
    namespace vegas {                                                                         \
    const void* name(int dim) {                                                               \
        static const void* const table[kFixedBinsMaxDim] = {                                  \
            VEGAS_NB(FN, 1), VEGAS_NB(FN, 2), VEGAS_NB(FN, 3), VEGAS_NB(FN, 4),                \
            VEGAS_NB(FN, 5), VEGAS_NB(FN, 6), VEGAS_NB(FN, 7), VEGAS_NB(FN, 8),                \
            VEGAS_NB(FN, 9), VEGAS_NB(FN, 10), VEGAS_NB(FN, 11), VEGAS_NB(FN, 12),             \
            VEGAS_NB(FN, 13), VEGAS_NB(FN, 14), VEGAS_NB(FN, 15), VEGAS_NB(FN, 16)};           \
        if (dim < 1 || dim > kFixedBinsMaxDim) return nullptr;                                \
        return table[dim - 1];                                                                \
    }                                                                                         \
    }
#define VEGAS_NB(FN, D) \
    (const void*)&vegas::vegas_iterate_kernel<float, D, FN, false, false, -1, vegas::kFixedBins>

#define VEGAS_KERNEL_TABLE(name, R, FN)                                                       \
    namespace vegas {                                                                         \
    const void* name(int dim, bool adapt) {                                                   \
        static const void* const table[kMaxDim][2] = {                                        \
            VEGAS_KERNEL_ROW(R, FN, 1),  VEGAS_KERNEL_ROW(R, FN, 2),  VEGAS_KERNEL_ROW(R, FN, 3),  \
            VEGAS_KERNEL_ROW(R, FN, 4),  VEGAS_KERNEL_ROW(R, FN, 5),  VEGAS_KERNEL_ROW(R, FN, 6),  \
            VEGAS_KERNEL_ROW(R, FN, 7),  VEGAS_KERNEL_ROW(R, FN, 8),  VEGAS_KERNEL_ROW(R, FN, 9),  \
            VEGAS_KERNEL_ROW(R, FN, 10), VEGAS_KERNEL_ROW(R, FN, 11), VEGAS_KERNEL_ROW(R, FN, 12), \
            VEGAS_KERNEL_ROW(R, FN, 13), VEGAS_KERNEL_ROW(R, FN, 14), VEGAS_KERNEL_ROW(R, FN, 15), \
            VEGAS_KERNEL_ROW(R, FN, 16), VEGAS_KERNEL_ROW(R, FN, 17), VEGAS_KERNEL_ROW(R, FN, 18), \
            VEGAS_KERNEL_ROW(R, FN, 19), VEGAS_KERNEL_ROW(R, FN, 20)};                        \
        if (dim < 1 || dim > kMaxDim) return nullptr;                                         \
        return table[dim - 1][adapt ? 1 : 0];                                                 \
    }                                                                                         \
    }
