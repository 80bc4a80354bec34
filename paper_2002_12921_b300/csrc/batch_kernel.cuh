// Many Vegas integrals in one persistent launch (the batch API of vegas.h).
//
// Work queue: the host cuts every integral's samples of an iteration into
// tiles (integral b, first sample, count).  Each thread block repeatedly takes
// the next tile index from an atomic ticket -- there is no waiting on other
// blocks -- stages that integral's grid in shared memory, runs the shared
// sample loop (integral_id = b in the Philox counter) and adds the tile's
// sums and histogram to integral b's accumulators with FP64 atomics.  The
// batch's integrals share one built-in integrand (a template parameter), each
// with its own parameters and box in its FnConsts.  A
// second, small launch refines every (integral, dimension) row and records
// each integral's estimate (batch.cu).
#pragma once

#include "iterate_kernel.cuh"
#include "vegas_internal.h"

namespace vegas {

struct BatchTile {
    unsigned b;                // integral
    unsigned count;            // samples in the tile
    unsigned long long start;  // first sample index
};

struct BatchInfo {
    int dim;
    int pad;
    unsigned long long n;         // samples per iteration
    unsigned long long edge_off;  // offset of the grid rows in `edges`
    unsigned long long hist_off;  // offset of the histogram rows in `hist`
};

struct BatchArgs {
    const BatchTile* tiles;
    const BatchInfo* info;
    const FnConsts* consts;  // per integral (Eq. 1 staging and prefactors)
    double* edges;
    double* hist;
    double* acc;             // per integral: S1, S2, nonfinite, unused
    unsigned* ctrl;          // ticket
    unsigned num_tiles;
    unsigned iter;
    int nbins;
    int max_dim;
    int hist_log2r;
    const float2* staged32;  // float path: staged pairs of every row (hist layout), else null
    unsigned rk0[10], rk1[10];
    int rowoff[kMaxDim];     // k N: row offsets of the staged grid (fill_row_offsets)
};

// One tile of integral b with compile-time dimension D and integrand FN.
// LOGR >= 0: the tile's histogram copies as a compile-time 2^LOGR (the
// big-block kernel always runs 32); -1: chosen per tile below.
template <typename R, int D, int FN, bool ADAPT, int LOGR = -1>
__device__ __forceinline__ void batch_tile(const BatchArgs& a, const BatchTile& t,
                                           typename Prec<R>::Pair* sgrid,
                                           typename Prec<R>::Hist* shist, double* sred,
                                           unsigned* sbad) {
    const int N = a.nbins;
    // Histogram copies: the shared memory is sized for the widest integral
    // with 2^hist_log2r copies; a tile of fewer dimensions takes as many
    // copies as fit in it, up to one per lane (lanes of a warp that share a
    // copy make the shared atomics retry).
    int logr = 0;
    if (ADAPT && LOGR >= 0) {
        logr = LOGR;
    } else if (ADAPT) {
        logr = a.hist_log2r;
        while (logr < 5 && (D << (logr + 1)) <= (a.max_dim << a.hist_log2r)) ++logr;
    }
    const FnConsts& fc = a.consts[t.b];
    const BatchInfo info = a.info[t.b];
    stage_grid<R, D, ADAPT>(a.edges + info.edge_off, N, logr, fc, sgrid, shist,
                            a.staged32 ? a.staged32 + info.hist_off : nullptr);
    R n4, nlast;
    jacobian_factors<R, D>(N, n4, nlast);
    __syncthreads();

    IterateSink<R, D, ADAPT, ADAPT ? LOGR : -1> sink(shist, N, logr);
    bool checks_ok = sample_loop<R, D, Integrand<R, FN>>(
        t.start + threadIdx.x, t.start + t.count, blockDim.x, a.iter, t.b << 8, a.rk0, a.rk1,
        fc, N, a.rowoff, (R)(sizeof(R) == 4 ? fc.C32 : fc.C), n4, nlast, sgrid, sink);
#ifdef VEGAS_DEBUG_CHECKS
    checks_ok &= edges_ok(a.edges + info.edge_off, D, N);
#endif
    report_checks(checks_ok, a.ctrl);

    const double s1 = sink.acc.block1(reinterpret_cast<FloatFloat*>(sred));
    const double s2 = sink.acc.block2(reinterpret_cast<FloatFloat*>(sred));
    const unsigned bad = block_sum(sink.bad, sbad);
    if (ADAPT) {
        __syncthreads();
        flush_hist(shist, D * N, logr, 1.0, a.hist + info.hist_off);
    }
    if (threadIdx.x == 0) {
        double* acc = a.acc + 4 * (size_t)t.b;
        atomicAdd(acc + 0, s1);
        atomicAdd(acc + 1, s2);
        if (bad) atomicAdd(acc + 2, (double)bad);
    }
    __syncthreads();  // the next tile restages the shared memory
}

// BOUND: the largest block the instantiation launches with (its launch
// bound): 256 (blocks of 32..256 threads), 512 (257..512), or kBigBlockThreads
// for one block per SM (float adapting rounds whose 32 histogram copies for the
// widest integral miss the default budget but fit that block).
template <typename R, int FN, bool ADAPT, int BOUND = 256>
__global__ void __launch_bounds__(BOUND) batch_iterate_kernel(const BatchArgs a) {
    using P = Prec<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sred[32];
    __shared__ unsigned sbad[32];
    __shared__ unsigned s_tile;
    typename P::Pair* sgrid = reinterpret_cast<typename P::Pair*>(smem_raw);
    typename P::Hist* shist = reinterpret_cast<typename P::Hist*>(sgrid + a.max_dim * a.nbins);

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctrl[kTicket], 1u);
        __syncthreads();
        const unsigned ti = s_tile;
        if (ti >= a.num_tiles) break;
        const BatchTile t = a.tiles[ti];
        switch (a.info[t.b].dim) {
#define VEGAS_BATCH_CASE(D) \
    case D:                                                                        \
        batch_tile<R, D, FN, ADAPT, BOUND == kBigBlockThreads ? 5 : -1>(a, t, sgrid, shist, \
                                                                       sred, sbad);   \
        break;
            VEGAS_BATCH_CASE(1) VEGAS_BATCH_CASE(2) VEGAS_BATCH_CASE(3) VEGAS_BATCH_CASE(4)
            VEGAS_BATCH_CASE(5) VEGAS_BATCH_CASE(6) VEGAS_BATCH_CASE(7) VEGAS_BATCH_CASE(8)
            VEGAS_BATCH_CASE(9) VEGAS_BATCH_CASE(10) VEGAS_BATCH_CASE(11) VEGAS_BATCH_CASE(12)
            VEGAS_BATCH_CASE(13) VEGAS_BATCH_CASE(14) VEGAS_BATCH_CASE(15) VEGAS_BATCH_CASE(16)
            VEGAS_BATCH_CASE(17) VEGAS_BATCH_CASE(18) VEGAS_BATCH_CASE(19) VEGAS_BATCH_CASE(20)
#undef VEGAS_BATCH_CASE
            default: __syncthreads(); break;
        }
    }
}

// the batch iterate kernel of a precision and built-in integrand for blocks of
// `block` threads (<= 512), for the host (batch_f32.cu / batch_f64.cu; nullptr
// for an integrand it lacks)
const void* batch_iterate_kernel_f32(int integrand, bool adapt, int block);
const void* batch_iterate_kernel_f64(int integrand, bool adapt, int block);
// the float big-block adapting kernel of an integrand (batch_f32.cu)
const void* batch_iterate_kernel_f32_big(int integrand);

}  // namespace vegas

// One (precision, integrand) pair's kernels, both adapt flags and both launch
// bounds, as the function NAME(adapt, block) (one source file each, so that
// they compile in parallel).
#define VEGAS_BATCH_TABLE(NAME, R, FN)                                                   \
    namespace vegas {                                                                    \
    const void* NAME(bool adapt, int block) {                                            \
        if (block > 256)                                                                 \
            return adapt ? (const void*)&batch_iterate_kernel<R, FN, true, 512>          \
                         : (const void*)&batch_iterate_kernel<R, FN, false, 512>;        \
        return adapt ? (const void*)&batch_iterate_kernel<R, FN, true>                   \
                     : (const void*)&batch_iterate_kernel<R, FN, false>;                 \
    }                                                                                    \
    }

// The float big-block adapting kernel of one integrand, as NAME().
#define VEGAS_BATCH_TABLE_BIG(NAME, FN)                                         \
    namespace vegas {                                                           \
    const void* NAME() {                                                        \
        return (const void*)&batch_iterate_kernel<float, FN, true, kBigBlockThreads>; \
    }                                                                           \
    }
