/*
 * vegas.h -- C ABI of the B300 (sm_103a) Vegas hot path.
 *
 * One Vegas iteration (VegasFlow, Sec. 2.2: the per-event step, then the
 * after-iteration refinement; the method is Lepage's, cited in Sec. 1):
 *   vegas_iterate  draws n samples from counter-based Philox4x32-10, maps them
 *                  through the adaptive grid, evaluates the integrand and
 *                  reduces sum fJ, sum (fJ)^2 and the per-dimension per-bin
 *                  (fJ)^2 histogram -- one fused kernel;
 *   vegas_refine   smooths, damps and re-partitions the grid from the
 *                  histogram -- one small kernel, device only;
 *   vegas_result   combines the iterations (inverse-variance weights) on the
 *                  host.
 *
 * Memory and streams.  The caller owns all device memory: it passes one
 * workspace buffer of vegas_workspace_bytes() bytes (any allocator; 256-byte
 * aligned) and a CUDA stream (cudaStream_t as void*, NULL = legacy default
 * stream).  The library never allocates device memory.  It owns only the small
 * host-side descriptor returned by vegas_init_grid.  Every call that launches
 * work is asynchronous on the stream; vegas_result, vegas_get_* synchronise it.
 *
 * Errors.  Every function returns a status (VEGAS_OK = 0).  No C++ exception
 * and no abort crosses the ABI.  Asynchronous device errors surface at the next
 * synchronising call.  A state whose call failed with VEGAS_ECUDA should be
 * destroyed.
 *
 * Sample counters.  Sample i (0-based, 64-bit, counted across launches of one
 * iteration) of iteration t draws Philox4x32-10 under key (seed low word, seed
 * high word) at counter (i low, i high, q | integral_id << 8, t) for
 * q = 0 .. ceil(dim/4)-1; dimension k takes word k mod 4 of call q = k/4.  The
 * result is therefore a pure function of (seed, grid, n, t), independent of
 * launch configuration and chunking.
 *
 * Bin and position.  For word w: bin j = floor(w N / 2^32) (exact integer),
 * position l = (w N) mod 2^32.  FP64 mode: frac = (l + 1/2) 2^-32.  FP32 mode:
 * frac = (floor(l / 2^9) + 1/2) 2^-23.  x = e_j + frac (e_{j+1} - e_j),
 * J = prod_k N (e_{j+1} - e_j).  In FP32 mode each bin's (start, width) pair --
 * already in the integrand's own coordinate -- is computed in double and
 * rounded once to float, and J uses the rounded width: inside every bin the map
 * is an exact change of variables (adjacent bins may overlap or leave a gap of
 * an ulp).
 *
 * Threads.  A state (or batch) is not thread-safe: calls on one state must not
 * run concurrently; different states may be used from different host threads.
 * What the library shares between states (the pool of pinned log staging, the
 * prepared launch shapes of its kernels) is guarded internally.
 *
 * Devices.  A workspace may live on any CUDA device of ordinal below 64
 * (VEGAS_MAX_DEVICES); launches on others fail with VEGAS_ECUDA, and
 * vegas_iterate_noalloc refuses them with VEGAS_EINVAL.
 *
 * CUDA graphs.  vegas_iterate and vegas_refine only enqueue kernels (no host
 * synchronisation), so a schedule of them can be captured from the state's
 * stream into a CUDA graph.  The iteration number, the log row it fills and the
 * float path's pre-scale are read from the state's device memory, not baked
 * into the launch: every replay runs the captured schedule as further
 * iterations (fresh Philox counters) from the grid it finds, appending to the
 * log.  Replays do not advance the host's iteration count, so the log's
 * capacity is enforced on the device: an iteration past max_iters does nothing
 * and makes vegas_result return VEGAS_ESTATE.  vegas_set_box, vegas_shard_*
 * and vegas_export_state rely on the host count; do not mix them with replays.
 */
#ifndef VEGAS_B300_VEGAS_H
#define VEGAS_B300_VEGAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define VEGAS_OK 0
#define VEGAS_EINVAL 1     /* an argument is out of range or NULL */
#define VEGAS_ECUDA 2      /* a CUDA runtime call failed (launch or sync) */
#define VEGAS_ENONFINITE 3 /* some f*J was NaN or infinite (left out of the sums) */
#define VEGAS_ESTATE 4     /* call out of order, iteration log full, bad grid, or (debug
                              build) a failed device check */
#define VEGAS_ENOSPACE 5   /* workspace smaller than vegas_workspace_bytes() */

/* ---- precision modes ---------------------------------------------------- */
#define VEGAS_FP64 0      /* map, integrand and sums in double */
#define VEGAS_FP32_EVAL 1 /* map and integrand in float; per-thread compensated
                             (Kahan) float sums, double above the thread; grid,
                             histogram, refinement and combination in double */

/* ---- built-in integrands over [0,1]^dim (VegasFlow Sec. 3.1) ------------- */
/* VEGAS_GAUSS      Eq. 1, per-dimension centres:
 *                  f = (a sqrt(pi))^-d exp(-sum_k (x_k - mu_k)^2 / a^2);
 *                  params = [a, mu_1 .. mu_d]            (nparams = 1 + d)
 *                  integral = prod_k (erf((1-mu_k)/a) + erf(mu_k/a)) / 2.
 * VEGAS_GAUSS_MIX2 (G(x; muA, a) + G(x; muB, a)) / 2 with G the Eq. 1 term;
 *                  params = [a, muA_1 .. muA_d, muB_1 .. muB_d] (1 + 2d).
 * VEGAS_FLAT       f = 1; params ignored (nparams may be 0).
 * VEGAS_GENZ_DISC  Eq. 2 normalised to integrate to 1: 0 if any x_k <= a_k,
 *                  else exp(sum_k c_k x_k) / prod_k (e^{c_k} - e^{c_k a_k})/c_k;
 *                  params = [a_1 .. a_d, c_1 .. c_d] (2d), c_k != 0.
 * VEGAS_GENZ_PPEAK Eq. 3 normalised to integrate to 1:
 *                  prod_k 1/(c_k^-2 + (x_k - a_k)^2) / (c_k (atan(c_k (1-a_k)) +
 *                  atan(c_k a_k))); params = [a_1 .. a_d, c_1 .. c_d] (2d), c_k > 0. */
#define VEGAS_GAUSS 0
#define VEGAS_GAUSS_MIX2 1
#define VEGAS_FLAT 2
#define VEGAS_GENZ_DISC 3
#define VEGAS_GENZ_PPEAK 4
/* VEGAS_USER       an integrand compiled by the caller (include/vegas_user_integrand.cuh),
 *                  attached with vegas_set_user_integrand before the first
 *                  iteration; params ignored. */
#define VEGAS_USER 5

/* ---- debug build ---------------------------------------------------------- */
/* libvegas_b300_debug.so (the same sources built with VEGAS_DEBUG_CHECKS) adds
 * device checks to the iterate kernels: every block checks the state's grid
 * (per dimension 0 and 1 at the ends, finite, strictly increasing edges) and
 * every sample its bin index (< nbins) and mapped coordinate (finite).  A failed check sets a
 * bit of the state's device status word; vegas_result, vegas_get_iterations
 * and the batch result calls then return VEGAS_ESTATE.  Nothing traps. */

/* ---- limits --------------------------------------------------------------- */
#define VEGAS_MAX_DIM 20
#define VEGAS_MAX_BINS 1024
#define VEGAS_MAX_DIM_X_BINS 8192 /* dim * nbins (shared-memory grid copy) */
#define VEGAS_MAX_DEVICES 64      /* device ordinals a workspace may live on */

typedef struct vegas_state vegas_state; /* opaque host descriptor */

/* Launch configuration; zeros select the defaults.  Under the defaults, a
 * float adapting iteration whose 32 per-lane histogram copies exceed the
 * default shared-memory budget (dim * nbins > 416) but fit one block runs as
 * one 768-thread block per SM instead (the same occupancy, no shared copies);
 * setting block_threads or blocks_per_sm keeps the configured shape. */
typedef struct {
    int block_threads;    /* threads per block of the iterate kernel (multiple of 32,
                             32 .. 256); default 256 */
    int blocks_per_sm;    /* resident blocks per SM the grid is sized for; default:
                             the occupancy limit */
    int min_samples_per_thread; /* the grid shrinks so that every thread gets at least
                                   this many samples; default 8 */
    uint64_t chunk_samples;     /* samples per launch inside one iteration; 0 = one
                                   launch per iteration */
} vegas_config;

/* Bytes of device workspace for a state of this shape with room for max_iters
 * iterations in its device log.  dim in [1, 20], nbins in [1, 1024],
 * dim*nbins <= 8192, max_iters >= 1.  Returns VEGAS_EINVAL otherwise. */
int vegas_workspace_bytes(int dim, int nbins, int max_iters, size_t *bytes);

/* Create a state: uniform grid e_l = l/nbins in every dimension (Lepage 1978,
 * Sec. 2: the starting grid), zero histogram, empty iteration log.
 *   mode       VEGAS_FP64 or VEGAS_FP32_EVAL
 *   integrand  one of the VEGAS_* integrand ids, params as documented above
 *              (copied; the caller may free them on return)
 *   d_workspace, ws_bytes  device buffer owned by the caller; it must outlive
 *              the state and must not be used by anything else meanwhile
 *   cuda_stream  the stream all work of this state is ordered on
 * On success *out receives the descriptor, which holds a small pinned host
 * buffer (the control words and up to 4096 log rows) through which every
 * later read of the log goes: taken from the library's process-wide pool of
 * page-locked blocks that destroyed states returned, else allocated with
 * cudaHostAlloc; VEGAS_ECUDA if it cannot be had.  Thread-safe.
 * Asynchronous: the workspace is initialised by work enqueued on the stream. */
int vegas_init_grid(vegas_state **out, int dim, int nbins, uint64_t seed, int mode, int integrand,
                    const double *params, int nparams, int max_iters, void *d_workspace,
                    size_t ws_bytes, void *cuda_stream);

/* Integrate over the box [lo_k, hi_k] (dim doubles each, finite, hi > lo)
 * instead of the unit cube: the grid stays in unit coordinates u, the integrand
 * is evaluated at x = lo + (hi - lo) u and the Jacobian gains prod (hi - lo).
 * The integrand's parameters keep their meaning in x (e.g. the Gaussian's
 * centres and width); a caller-compiled integrand receives x.  Only before the
 * first iteration (else VEGAS_ESTATE); VEGAS_EINVAL on a bad box.  States with a
 * box are checkpointed with it, and vegas_gauss_adjoint differentiates the
 * boxed integral. */
int vegas_set_box(vegas_state *s, const double *lo, const double *hi);

/* Change the launch configuration (cfg == NULL restores the defaults). */
int vegas_set_config(vegas_state *s, const vegas_config *cfg);

/* Run one iteration of n_samples >= 2 samples (at most VEGAS_MAX_SAMPLE_INDEX)
 * on the current grid (the per-event step of Sec. 2.2).  adapt != 0 also adds each sample's (fJ)^2 to
 * the histogram bin of each dimension for the next vegas_refine.  Appends
 * (S1, S2, n, nonfinite, I = S1/n, var = (S2/n - I^2)/(n-1)) to the device log.
 * Asynchronous; VEGAS_ESTATE if the log is full. */
int vegas_iterate(vegas_state *s, uint64_t n_samples, int adapt);

/* Sample indices stay below this bound (2^64 - 2^33) in every call that takes
 * them (n_samples, n_total, i0 + n): a thread's next index then never wraps
 * around 2^64.  Larger values return VEGAS_EINVAL. */
#define VEGAS_MAX_SAMPLE_INDEX 0xFFFFFFFE00000000ull

/* Refine the grid from the accumulated histogram and clear it (the
 * after-iteration step of Sec. 2.2; Lepage 1978 Sec. 3 and the 1980 report):
 * per dimension, three-point smoothing (the two end bins averaged with their
 * one neighbour), normalisation r_j = h_j / sum h, damping
 * m_j = ((r_j - 1)/ln r_j)^alpha, and new edges where the piecewise-linear
 * cumulative m reaches l * sum(m)/N, l = 1..N-1.  A dimension whose histogram
 * sums to 0 or is not finite keeps its grid.  alpha >= 0.  Device only,
 * asynchronous. */
int vegas_refine(vegas_state *s, double alpha);

/* Combine iterations first_iter .. n_iter-1 (inverse-variance weighted mean,
 * sigma = (sum 1/var)^-1/2, chi^2 per degree of freedom; an iteration with
 * zero variance makes it the plain mean with sigma 0): the cumulative
 * estimate of Lepage 1978 Sec. 2, which VegasFlow reports as its value +-
 * error (Table 1).  The log is read through the descriptor's pinned host
 * staging.  Synchronises the
 * stream.  Any output pointer may be NULL.  Returns VEGAS_ENONFINITE (after
 * filling the outputs) if a combined iteration saw non-finite f*J. */
int vegas_result(vegas_state *s, int first_iter, double *mean, double *sigma, double *chi2_dof,
                 int *n_iter);

/* The same combination (Lepage 1978 Sec. 2's cumulative estimate) over
 * iterations first_iter .. end_iter-1 only (for the running result after each
 * iteration, as an integrator prints it per iteration).  VEGAS_EINVAL if end_iter <=
 * first_iter or iteration end_iter-1 is not logged.  Synchronises. */
int vegas_result_range(vegas_state *s, int first_iter, int end_iter, double *mean,
                       double *sigma, double *chi2_dof);

/* Copy the log to host memory: row t = {S1, S2, n, nonfinite, I, var} for
 * t < min(max_rows, n_iter).  Synchronises the stream. */
int vegas_get_iterations(vegas_state *s, double *host_rows, int max_rows, int *n_rows);

/* Device time of each logged iteration, in ns of the GPU's global timer: from
 * the start of the first block of its first launch to the end of its last
 * launch's reduction (launch gaps inside a chunked iteration included, launch
 * latency before it not); for a sharded iteration, this rank's own range.
 * host_ns: max_rows doubles; *n_rows receives the count.  Synchronises. */
int vegas_get_iteration_times(vegas_state *s, double *host_ns, int max_rows, int *n_rows);

/* Copy the grid -- the adaptive map's bin edges e_{k,0..N} per dimension
 * (Lepage 1978 Sec. 3), which the after-iteration step of VegasFlow Sec. 2.2
 * refines -- (dim x (nbins+1) doubles, row-major) to / from host memory.
 * vegas_set_grid checks e_0 = 0, e_N = 1 and strict increase (VEGAS_ESTATE
 * otherwise).  Both synchronise the stream. */
int vegas_get_grid(vegas_state *s, double *host_edges);
int vegas_set_grid(vegas_state *s, const double *host_edges);

/* Copy the histogram (dim x nbins doubles) to host memory.  Synchronises. */
int vegas_get_histogram(vegas_state *s, double *host_hist);

/* Write the Philox4x32-10 words that samples i0 .. i0+n-1 of iteration iter
 * draw (the counter layout above) to d_out, n x dim uint32 rows in device
 * memory owned by the caller; the same device function the iterate kernel
 * uses.  A reproducibility and test aid.  dim in [1, 20], n at most
 * VEGAS_MAX_SAMPLE_INDEX, d_out device memory (else VEGAS_EINVAL);
 * asynchronous on the stream. */
int vegas_sample_words(uint64_t seed, uint32_t integral_id, uint32_t iter, uint64_t i0,
                       uint64_t n, int dim, uint32_t *d_out, void *cuda_stream);

/* ---- one integral sharded over several devices ---------------------------- */
/* Sample indices are global, so one iteration of n samples can be split into
 * contiguous ranges computed on different devices (each with its own state,
 * the same seed, grid and iteration count).  Per iteration, every rank:
 *   vegas_iterate_range(s, n, begin, end, adapt)   its samples [begin, end);
 *   vegas_shard_export(s, d_buf)                   packs its partial sums;
 *   (sum the buffers over the ranks, e.g. an all-reduce)
 *   vegas_shard_import(s, d_buf, n)                installs the totals;
 *   vegas_refine(s, alpha)                         identical on every rank.
 * The grids then stay identical across ranks and the log equals a single
 * device's run up to the order of the sums.  The exchanged buffer holds
 * 3 + dim*nbins doubles: {S1, S2, nonfinite, histogram (dim x nbins)}. */

/* Samples [i_begin, i_end) of an iteration of n_total samples (0 <= i_begin <
 * i_end <= n_total <= VEGAS_MAX_SAMPLE_INDEX).  The log row holds this range's sums until
 * vegas_shard_import replaces them.  Asynchronous. */
int vegas_iterate_range(vegas_state *s, uint64_t n_total, uint64_t i_begin, uint64_t i_end,
                        int adapt);
/* Copy the last iteration's {S1, S2, nonfinite} and the histogram into d_buf
 * (device, 3 + dim*nbins doubles).  Asynchronous.  Here and in
 * vegas_shard_import, vegas_gauss_adjoint and vegas_grid_digest, the
 * caller's buffer must be device memory on the state's device (cudaMalloc or
 * a framework's device allocation): anything else returns VEGAS_EINVAL before
 * anything is enqueued. */
int vegas_shard_export(vegas_state *s, double *d_buf);
/* Replace the last iteration's sums and the histogram by d_buf's totals and
 * recompute its I and var for n_total samples.  Asynchronous. */
int vegas_shard_import(vegas_state *s, const double *d_buf, uint64_t n_total);

/* Several fixed-grid iterations exchanged at once.  A fixed-grid iteration
 * changes neither the grid nor the histogram, and the combination (Lepage
 * 1978 Sec. 2) needs its totals only when the result is read, so the ranks may
 * run iterations first_iter .. first_iter+count-1 on their own ranges and sum
 * their rows in one reduction:
 *   vegas_shard_export_rows  copies each row's {S1, S2, nonfinite} into d_buf
 *                            (3*count device doubles, row by row);
 *   vegas_shard_import_rows  replaces the rows' sums by d_buf's totals and
 *                            recomputes each row's I and var for n_total
 *                            samples (the same n for every row).
 * The rows must be logged on the host (first_iter >= 0, count >= 1,
 * first_iter + count <= iterations enqueued; else VEGAS_ESTATE) and must be
 * fixed-grid iterations: an adapting iteration's histogram has to be
 * exchanged (vegas_shard_export / import) before its refinement.  Until the
 * import, a row holds the rank's own sums (and the float path's pre-scale of
 * the next iteration follows that partial estimate, which changes only the
 * float rounding).  Device buffers as for vegas_shard_export; asynchronous. */
int vegas_shard_export_rows(vegas_state *s, int first_iter, int count, double *d_buf);
int vegas_shard_import_rows(vegas_state *s, int first_iter, int count, const double *d_buf,
                            uint64_t n_total);

/* Gradient of the Eq. 1 Gaussian integral with respect to its parameters, by
 * the reparameterised fixed-grid estimator: on the state's current (frozen)
 * grid, sample i of iteration `iter` is regenerated from its Philox counter
 * (nothing per sample is stored), and
 *   I = (1/n) sum_i f(x_i) J_i,   dI/dtheta = (1/n) sum_i J_i df/dtheta(x_i),
 * with df/dmu_k = f 2 (x_k - mu_k)/a^2 and df/da = (f/a)(2 sum_k (x_k-mu_k)^2/a^2 - d).
 * params = [a, mu_1 .. mu_d] (as VEGAS_GAUSS; independent of the state's own
 * integrand).  d_out: 2 (dim+2) + 1 device doubles owned by the caller:
 * [I, dI/dmu_1 .. dI/dmu_d, dI/da, then the Monte Carlo variances of those
 * d+2 means, then the count of non-finite weights].  grad == 0 computes only
 * I and its variance (the other entries are set to 0).  Uses the state's
 * mode, seed, grid, workspace and stream; the same (iter, n) as an earlier
 * vegas_iterate on the same grid reproduces its samples exactly.
 * Over a box (vegas_set_box) the samples are x = lo + (hi - lo) u and this is
 * the gradient of the boxed integral.  Asynchronous.  The paper's integrator
 * has no gradient; this is the differentiable extension of the same
 * estimator. */
int vegas_gauss_adjoint(vegas_state *s, const double *params, int nparams, uint32_t iter,
                        uint64_t n_samples, int grad, double *d_out);

/* ---- many integrals in one persistent launch ------------------------------ */
/* A batch holds `count` independent integrals of one built-in integrand family
 * (Eq. 1 Gaussians with vegas_batch_init; any family, and a box per integral,
 * with vegas_batch_init_integrand), each of its own dimension (1..20), samples
 * per iteration and parameters, all with nbins bins per dimension, sharing one
 * seed and one iteration schedule.
 * Integral b draws its samples with integral_id = b in the counter (see the
 * top of this file), so its result equals that of a single vegas_state run
 * with the same grid, seed and iteration indices and integral id b.
 * vegas_batch_iterate enqueues one iteration of every integral as one
 * persistent launch -- thread blocks take (integral, sample range) tiles from
 * an atomic ticket, without waiting on each other -- followed by one launch
 * that refines every (integral, dimension) grid row and records each
 * integral's estimate.  Those launches take no host synchronisation, so a
 * whole schedule can be captured in a CUDA graph (vegas_batch_reset first,
 * then the iterations) and replayed.  The caller owns the device workspace
 * and the stream; the library copies the tile table and the per-integral
 * constants into the workspace at vegas_batch_init (and at
 * vegas_batch_set_config) with host-to-device copies ordered on the stream. */
typedef struct vegas_batch vegas_batch;

/* params: for integral b, [a_b, mu_b,1 .. mu_b,dims[b]], concatenated in
 * order (sum_b (1 + dims[b]) doubles).  tile_samples 0 = default (65536). */
int vegas_batch_workspace_bytes(int count, const int *dims, const uint64_t *n_samples,
                                int nbins, int max_iters, size_t *bytes);
int vegas_batch_init(vegas_batch **out, int count, const int *dims, const uint64_t *n_samples,
                     int nbins, uint64_t seed, int mode, const double *params, int max_iters,
                     void *d_workspace, size_t ws_bytes, void *cuda_stream);
/* The same for any built-in integrand (VEGAS_GAUSS .. VEGAS_GENZ_PPEAK, shared
 * by the batch; VEGAS_EINVAL for VEGAS_USER): params holds each integral's
 * parameters in that integrand's layout (VEGAS_GAUSS 1 + d, VEGAS_GAUSS_MIX2
 * 1 + 2d, VEGAS_GENZ_* 2d, VEGAS_FLAT none; params may be NULL when the total
 * is 0), concatenated in order.  box_lo, box_hi: NULL for the unit cube, else
 * each integral's box [lo_k, hi_k] (as vegas_set_box), dims[b] doubles per
 * integral concatenated in order (sum_b dims[b] each).  vegas_batch_init is
 * this call with VEGAS_GAUSS and no box. */
int vegas_batch_init_integrand(vegas_batch **out, int count, const int *dims,
                               const uint64_t *n_samples, int nbins, uint64_t seed, int mode,
                               int integrand, const double *params, const double *box_lo,
                               const double *box_hi, int max_iters, void *d_workspace,
                               size_t ws_bytes, void *cuda_stream);
/* Block size (32..512, multiple of 32) and samples per tile (>= 128, multiple
 * of 32; a tile of block size x s gives each thread s samples); 0 keeps the
 * current value.  Rebuilds the tile table.  At the default block size (256),
 * float adapting rounds run as one 768-thread block per SM when 32 histogram
 * copies for the widest integral need it and fit.  Results do not depend on
 * either (the samples are functions of their counters). */
int vegas_batch_set_config(vegas_batch *b, int block_threads, uint64_t tile_samples);
/* Samples per tile by dimension: tiles[d-1] for the integrals of dimension d
 * (d = 1 .. count, count <= VEGAS_MAX_DIM; each 0 = the vegas_batch_set_config
 * size, else >= 128 and a multiple of 32); tiles == NULL with count 0 clears
 * them.  Work per sample grows with the dimension, so smaller tiles for wide
 * integrals even out the blocks' loads.  Rebuilds the tile table; results do
 * not depend on it. */
int vegas_batch_set_tiles_by_dim(vegas_batch *b, const uint64_t *tiles, int count);
/* Order the batch's work on another stream (for graph capture on a side stream). */
int vegas_batch_set_stream(vegas_batch *b, void *cuda_stream);
/* Uniform grids, cleared histograms and logs, iteration counter 0 (device work
 * on the stream; no host synchronisation). */
int vegas_batch_reset(vegas_batch *b);
/* One iteration of every integral (adapt != 0: histograms and refinement with
 * damping alpha).  Asynchronous; VEGAS_ESTATE when max_iters is reached. */
int vegas_batch_iterate(vegas_batch *b, int adapt, double alpha);
/* Combined result of integral `index` over iterations first_iter .. done-1, as
 * vegas_result.  Synchronises the stream. */
int vegas_batch_result(vegas_batch *b, int index, int first_iter, double *mean, double *sigma,
                       double *chi2_dof, int *n_iter);
/* Log rows {S1, S2, n, nonfinite, I, var} of every integral: count x max_iters
 * x 6 doubles (rows past the iterations done are zero).  Synchronises. */
int vegas_batch_get_log(vegas_batch *b, double *host_rows);
/* Grid of integral `index`: dims[index] x (nbins+1) doubles.  Synchronises. */
int vegas_batch_get_grid(vegas_batch *b, int index, double *host_edges);
/* The (fJ)^2 histogram (Lepage 1978 Sec. 3's per-bin accumulator) that the
 * last adapting iteration of integral `index` refined its grid from:
 * dims[index] x nbins doubles (zeros before the first adapting iteration).
 * The batch keeps a copy of every row as it refines it (VegasFlow Sec. 2.3:
 * exporting histograms during integration).  Synchronises. */
int vegas_batch_get_histogram(vegas_batch *b, int index, double *host_hist);
int vegas_batch_destroy(vegas_batch *b);

/* ---- entry point for callers that cannot allocate device memory ---------- */
/* The paper has no counterpart to this call; it exists for callers that are not
 * allowed to allocate device memory -- code that runs inside a host framework
 * which owns every device allocation (a plug-in in someone else's process, an
 * embedded runtime with a fixed memory budget), or code that only holds the
 * buffers it was handed.  Such callers cannot provide the workspace the
 * vegas_init_grid path needs.
 *
 * vegas_iterate_noalloc runs one iteration of the VEGAS_GAUSS integrand
 * (params = [a, mu_1 .. mu_d]) on the grid d_edges (dim x (nbins+1) device
 * doubles) with the counters of iteration `iter`, writes
 * {S1, S2, n, nonfinite, I, var} to d_result (6 device doubles) and, when
 * adapt != 0, refines d_edges in place with damping alpha (the same kernels and
 * rules as vegas_iterate + vegas_refine).  It allocates nothing: its scratch
 * (block partials, a ticket word, the histogram) is one static device array of
 * VEGAS_NOALLOC_SCRATCH_BYTES bytes in the library, which every GPU that loads
 * the library holds until the process exits.
 *   - dim * nbins > VEGAS_NOALLOC_MAX_DIM_X_BINS returns VEGAS_ENOSPACE (the
 *     histogram would not fit the scratch); the launch never uses more than
 *     VEGAS_NOALLOC_MAX_BLOCKS blocks.
 *   - d_edges and d_result must be device memory of one device (else
 *     VEGAS_EINVAL, before anything is enqueued).
 *   - A call looks up the scratch's device address on that device
 *     (cudaGetSymbolAddress), afresh whenever its stream is not capturing, so
 *     a context torn down and rebuilt in between (cudaDeviceReset) is seen;
 *     make the first call on each device before any stream capture starts.
 *   - Every call shares the one scratch array and it keeps the last call's
 *     contents; each call clears what must start at zero.  Calls whose work
 *     overlaps on the GPU (other streams, other host threads) race on the
 *     scratch: order them on one stream.
 *   - In FP32 mode the sums are not pre-scaled by a previous estimate (there is
 *     none); the built-in integrand is normalised, so none is needed.
 * Asynchronous on the stream; n_samples in [2, 2^40]. */
#define VEGAS_NOALLOC_MAX_DIM_X_BINS 4096
#define VEGAS_NOALLOC_MAX_BLOCKS 2048
#define VEGAS_NOALLOC_SCRATCH_BYTES 98560
int vegas_iterate_noalloc(double *d_edges, int dim, int nbins, uint64_t seed, uint32_t iter,
                          int mode, const double *params, int nparams, uint64_t n_samples,
                          int adapt, double alpha, double *d_result, void *cuda_stream);

/* A 64-bit digest of the grid's bit patterns, for checking that the ranks
 * of a sharded integral hold identical grids after a refinement (the exchange
 * above keeps them equal only if every rank receives the same totals):
 *   digest = sum over the dim*(nbins+1) edges i (row-major) of
 *            bits(e_i) * (splitmix64(i) | 1)   mod 2^64,
 * splitmix64 being Vigna's SplitMix64 output function applied to i.  Equal
 * grids give equal digests; grids that differ in one edge's bits never do.
 * Writes {digest, ~digest} to d_out (2 uint64 of caller device memory, 8-byte
 * aligned): one all-reduce of the pair with MAX then yields the largest digest
 * and the complement of the smallest.  Asynchronous on the stream. */
int vegas_grid_digest(vegas_state *s, uint64_t *d_out);

/* ---- checkpoint / resume -------------------------------------------------- */
/* A state's resumable content as a flat little-endian blob -- what the
 * per-event and after-iteration steps of VegasFlow Sec. 2.2 carry from one
 * iteration to the next (the grid, the accumulated histogram, the
 * per-iteration estimates of Lepage 1978 Sec. 2-3); the paper itself
 * describes no checkpointing.  Contents: shape, mode,
 * integrand and its parameters, seed, iteration count, launch configuration,
 * the grid, the histogram (an adapting iteration not yet refined), the
 * iteration log and the box (vegas_set_box; format version 2, version-1 blobs
 * without a box are still read).  Because every sample is a function of (seed, iteration,
 * index), a state imported from a blob continues exactly as the exported one
 * would have.  Export synchronises the stream.  With buf == NULL, *bytes
 * receives the blob size; otherwise *bytes must hold at least that size. */
int vegas_export_state(vegas_state *s, void *buf, size_t *bytes);
/* Create a state from a blob of exactly `bytes` bytes (VEGAS_EINVAL if it is
 * malformed -- including a size other than its header implies and a grid
 * vegas_set_grid would refuse -- or of another
 * format version) on a caller workspace of at least vegas_workspace_bytes()
 * for the blob's shape and iteration capacity.  Asynchronous on the stream. */
int vegas_import_state(vegas_state **out, const void *buf, size_t bytes, void *d_workspace,
                       size_t ws_bytes, void *cuda_stream);

/* ---- user-supplied integrands (VegasFlow Sec. 2.3: integrands written in
 * C++ or CUDA and linked into the integrator) ------------------------------- */
/* The kernels of an integrand compiled in the caller's own CUDA translation
 * unit by the VEGAS_USER_INTEGRAND macro of include/vegas_user_integrand.cuh,
 * which returns a pointer to this descriptor.  The library never launches
 * the caller's kernels itself: it sizes the launch with `prepare` and issues
 * it through `launch`, both code of the caller's module (so the kernels need
 * not be registered with the library's CUDA runtime).
 *   dim         the dimension the kernels were compiled for
 *   args_bytes  the size of the kernels' argument block, checked against the
 *               library's own (a mismatch means the two were built from
 *               different headers)
 *   prepare     for (mode, adapt, block threads, dynamic shared bytes): raise
 *               the kernel's shared-memory limit if needed (to the device's
 *               maximum for the kernel, never lower) and store its resident
 *               blocks per SM in *blocks; returns a cudaError_t value.  The
 *               state calls it on its first fixed-grid and first adapting
 *               iteration and keeps the answer
 *   launch      enqueue the kernel of (mode, adapt) with the argument block
 *               `args` on `stream`; returns a cudaError_t value */
typedef struct {
    int dim;
    size_t args_bytes;
    int (*prepare)(int mode, int adapt, int block, size_t smem, int *blocks);
    int (*launch)(int mode, int adapt, const void *args, unsigned grid, unsigned block,
                  size_t smem, void *stream);
} vegas_user_integrand;

/* Attach user kernels to a state created with integrand VEGAS_USER (the
 * descriptor is copied; d_data is a device pointer, owned by the caller and
 * kept alive while the state iterates, handed unchanged to every evaluation
 * of the integrand; it may be NULL).  The state then iterates, refines,
 * shards and checkpoints as with a built-in integrand; a state restored by
 * vegas_import_state needs the call again.  VEGAS_EINVAL if the state is not
 * VEGAS_USER, the dimension or the argument-block size differ, or a callback
 * is NULL.  Iterating a VEGAS_USER state without it returns VEGAS_ESTATE. */
int vegas_set_user_integrand(vegas_state *s, const vegas_user_integrand *u, const void *d_data);


/* ---- measurement: pipe peaks ---------------------------------------------- */
/* The peak rate of one operation the iterate kernels depend on, measured on
 * the current device: every SM filled with blocks whose threads each run 8
 * independent chains of the operation for `iters` steps (0: a default of about
 * a millisecond per launch), one warm-up launch, then one launch timed with
 * CUDA events on the stream.  out[0] = lane-operations per second, out[1] = the
 * SM clock during the timed launch in MHz (cycle counter over global timer,
 * read by one block), out[2] = SM count, out[3] = blocks launched.  d_scratch:
 * caller device memory of at least VEGAS_PIPE_SCRATCH_BYTES, 8-byte aligned.
 * Synchronises the stream.  VEGAS_EINVAL for an unknown op or a bad argument,
 * VEGAS_ECUDA if a launch fails. */
#define VEGAS_PIPE_FFMA 0      /* float fused multiply-add */
#define VEGAS_PIPE_DFMA 1      /* double fused multiply-add */
#define VEGAS_PIPE_EX2 2       /* ex2.approx.ftz.f32 */
#define VEGAS_PIPE_PRODUCT 3   /* 32x32 -> 64-bit product as umulhi + low multiply */
#define VEGAS_PIPE_IMAD 4      /* 32-bit multiply-add, low word */
#define VEGAS_PIPE_LDS 5       /* 32-bit shared-memory load, conflict free */
#define VEGAS_PIPE_ATOMS_U32 6 /* 32-bit integer atomic add to shared memory */
#define VEGAS_PIPE_ATOMS_F32 7 /* float atomic add to shared memory */
#define VEGAS_PIPE_COUNT 8
#define VEGAS_PIPE_SCRATCH_BYTES 64
int vegas_pipe_peak(int op, uint32_t iters, void *d_scratch, size_t scratch_bytes,
                    void *cuda_stream, double *out);

/* ---- fault injection (testing) ------------------------------------------- */
/* Make the countdown-th of this state's next enqueueing calls (vegas_iterate,
 * vegas_iterate_range, vegas_refine; 1 = the next one) return VEGAS_ECUDA
 * before it enqueues or changes anything, as a failed launch would, so that a
 * caller's error handling and recovery can be tested without a GPU fault.
 * countdown 0 cancels.  Host-side only.  VEGAS_EINVAL for countdown < 0. */
int vegas_inject_failure(vegas_state *s, int countdown);

/* Release the descriptor (not the caller's workspace); its pinned host
 * staging goes back to the library's pool (at most 64 blocks wait there; the
 * rest are freed).  Synchronises the stream first.  NULL is accepted. */
int vegas_destroy(vegas_state *s);

/* Static text for a status code. */
const char *vegas_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* VEGAS_B300_VEGAS_H */
