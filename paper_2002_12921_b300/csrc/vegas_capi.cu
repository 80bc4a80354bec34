// Host side of the C ABI declared in include/vegas.h: argument checks,
// workspace layout, integrand constants, launch configuration, and the
// host-side combination of iterations.
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "philox.cuh"
#include "vegas_internal.h"

namespace vegas {
const void* iterate_table_f32_gauss(int dim, bool adapt);
const void* iterate_table_f32_mix2(int dim, bool adapt);
const void* iterate_table_f32_flat(int dim, bool adapt);
const void* iterate_table_f32_genz_disc(int dim, bool adapt);
const void* iterate_table_f32_genz_ppeak(int dim, bool adapt);
const void* iterate_table_f64_gauss(int dim, bool adapt);
const void* iterate_table_f64_mix2(int dim, bool adapt);
const void* iterate_table_f64_flat(int dim, bool adapt);
const void* iterate_table_f64_genz_disc(int dim, bool adapt);
const void* iterate_table_f64_genz_ppeak(int dim, bool adapt);

const void* iterate_kernel_f32(int integrand, int dim, bool adapt) {
    switch (integrand) {
    case VEGAS_GAUSS: return iterate_table_f32_gauss(dim, adapt);
    case VEGAS_GAUSS_MIX2: return iterate_table_f32_mix2(dim, adapt);
    case VEGAS_FLAT: return iterate_table_f32_flat(dim, adapt);
    case VEGAS_GENZ_DISC: return iterate_table_f32_genz_disc(dim, adapt);
    case VEGAS_GENZ_PPEAK: return iterate_table_f32_genz_ppeak(dim, adapt);
    default: return nullptr;
    }
}

const void* iterate_table_big_f32_gauss(int dim);
const void* iterate_table_big_f32_mix2(int dim);
const void* iterate_table_big_f32_flat(int dim);
const void* iterate_table_big_f32_genz_disc(int dim);
const void* iterate_table_big_f32_genz_ppeak(int dim);

const void* iterate_kernel_f32_big(int integrand, int dim) {
    switch (integrand) {
    case VEGAS_GAUSS: return iterate_table_big_f32_gauss(dim);
    case VEGAS_GAUSS_MIX2: return iterate_table_big_f32_mix2(dim);
    case VEGAS_FLAT: return iterate_table_big_f32_flat(dim);
    case VEGAS_GENZ_DISC: return iterate_table_big_f32_genz_disc(dim);
    case VEGAS_GENZ_PPEAK: return iterate_table_big_f32_genz_ppeak(dim);
    default: return nullptr;
    }
}

const void* iterate_table_few_f32_gauss(int dim);
const void* iterate_table_few_f32_mix2(int dim);
const void* iterate_table_few_f32_flat(int dim);
const void* iterate_table_few_f32_genz_disc(int dim);
const void* iterate_table_few_f32_genz_ppeak(int dim);

const void* iterate_kernel_f32_few(int integrand, int dim) {
    switch (integrand) {
    case VEGAS_GAUSS: return iterate_table_few_f32_gauss(dim);
    case VEGAS_GAUSS_MIX2: return iterate_table_few_f32_mix2(dim);
    case VEGAS_FLAT: return iterate_table_few_f32_flat(dim);
    case VEGAS_GENZ_DISC: return iterate_table_few_f32_genz_disc(dim);
    case VEGAS_GENZ_PPEAK: return iterate_table_few_f32_genz_ppeak(dim);
    default: return nullptr;
    }
}

const void* iterate_table_nb_f32_gauss(int dim);
const void* iterate_table_nb_f32_mix2(int dim);
const void* iterate_table_nb_f32_flat(int dim);
const void* iterate_table_nb_f32_genz_disc(int dim);
const void* iterate_table_nb_f32_genz_ppeak(int dim);

const void* iterate_kernel_f32_nb(int integrand, int dim) {
    switch (integrand) {
    case VEGAS_GAUSS: return iterate_table_nb_f32_gauss(dim);
    case VEGAS_GAUSS_MIX2: return iterate_table_nb_f32_mix2(dim);
    case VEGAS_FLAT: return iterate_table_nb_f32_flat(dim);
    case VEGAS_GENZ_DISC: return iterate_table_nb_f32_genz_disc(dim);
    case VEGAS_GENZ_PPEAK: return iterate_table_nb_f32_genz_ppeak(dim);
    default: return nullptr;
    }
}

const void* iterate_kernel_f64(int integrand, int dim, bool adapt) {
    switch (integrand) {
    case VEGAS_GAUSS: return iterate_table_f64_gauss(dim, adapt);
    case VEGAS_GAUSS_MIX2: return iterate_table_f64_mix2(dim, adapt);
    case VEGAS_FLAT: return iterate_table_f64_flat(dim, adapt);
    case VEGAS_GENZ_DISC: return iterate_table_f64_genz_disc(dim, adapt);
    case VEGAS_GENZ_PPEAK: return iterate_table_f64_genz_ppeak(dim, adapt);
    default: return nullptr;
    }
}

int hist_log2r(int mode, int dim, int nbins) {
    const size_t hist = mode == VEGAS_FP32_EVAL ? sizeof(float) : sizeof(double);
    int lr = 5;
    while (lr > 0 && ((size_t)dim * nbins * hist << lr) > kHistCopyBudget) --lr;
    return lr;
}

size_t iterate_smem_bytes(int mode, int dim, int nbins, bool adapt, int log2r) {
    const size_t pair = mode == VEGAS_FP32_EVAL ? 2 * sizeof(float) : 2 * sizeof(double);
    const size_t hist = mode == VEGAS_FP32_EVAL ? sizeof(float) : sizeof(double);
    return (size_t)dim * nbins * (pair + (adapt ? hist << log2r : 0));
}

namespace {
bool finite_params(const double* p, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}
}  // namespace

// Integrand constants for both precisions (see FnConsts).  Index 0 of the
// staging transform is the double path, index 1 the float path.
int make_consts(int integrand, int dim, int nbins, const double* params, int nparams,
                FnConsts* fc) {
    std::memset(fc, 0, sizeof(*fc));
    const double log2e = 1.4426950408889634;
    const double npow = std::pow((double)nbins, dim);  // N^dim of the FP64 Jacobian
    for (int k = 0; k < dim; ++k) fc->sc[0][k] = fc->sc[1][k] = 1.0;
    switch (integrand) {
    case VEGAS_GAUSS:
    case VEGAS_GAUSS_MIX2: {
        const int need = integrand == VEGAS_GAUSS ? 1 + dim : 1 + 2 * dim;
        if (!params || nparams < need || !finite_params(params, need)) return VEGAS_EINVAL;
        const double a = params[0];
        if (!(a > 0.0)) return VEGAS_EINVAL;
        // (a sqrt(pi))^-d, halved for the two-term mixture
        double norm = std::pow(a * std::sqrt(M_PI), -(double)dim);
        if (integrand == VEGAS_GAUSS_MIX2) norm *= 0.5;
        // double: z = (x - mu)/a, f ~ exp(-sum z^2); float: z = kappa (x - mu),
        // kappa^2 = log2(e)/a^2, f ~ 2^(-sum z^2)
        const double kappa = std::sqrt(log2e) / a;
        for (int k = 0; k < dim; ++k) {
            const double mu = params[1 + k];
            fc->sc[0][k] = 1.0 / a;
            fc->sh[0][k] = -mu / a;
            fc->sc[1][k] = kappa;
            fc->sh[1][k] = -mu * kappa;
            if (integrand == VEGAS_GAUSS_MIX2) {
                const double dmu = mu - params[1 + dim + k];  // z_B = z_A + (mu_A - mu_B) sc
                fc->d64[k] = dmu / a;
                fc->d32[k] = (float)(dmu * kappa);
            }
        }
        fc->C = norm * npow * std::pow(a, dim);
        fc->C32 = norm / std::pow(kappa, dim);
        return VEGAS_OK;
    }
    case VEGAS_FLAT:
    case VEGAS_USER:  // identity staging: the caller's integrand sees x itself
        fc->C = npow;
        fc->C32 = 1.0;
        return VEGAS_OK;
    case VEGAS_GENZ_DISC: {
        if (!params || nparams < 2 * dim || !finite_params(params, 2 * dim)) return VEGAS_EINVAL;
        double norm = 1.0;  // prod_k (e^{c_k} - e^{c_k a_k}) / c_k
        for (int k = 0; k < dim; ++k) {
            const double ak = params[k], ck = params[dim + k];
            if (ck == 0.0) return VEGAS_EINVAL;
            norm *= (std::exp(ck) - std::exp(ck * ak)) / ck;
            fc->t64[k] = ak;
            fc->d64[k] = ck;
            fc->t32[k] = (float)ak;
            fc->d32[k] = (float)(ck * log2e);
        }
        if (!(norm > 0.0) || !std::isfinite(norm)) return VEGAS_EINVAL;
        fc->C = npow / norm;
        fc->C32 = 1.0 / norm;
        return VEGAS_OK;
    }
    case VEGAS_GENZ_PPEAK: {
        if (!params || nparams < 2 * dim || !finite_params(params, 2 * dim)) return VEGAS_EINVAL;
        // z = c (x - a): 1/(c^-2 + (x-a)^2) = c^2/(1 + z^2); with the staging's
        // 1/prod c the prefactor is prod_k c_k / integral_k
        double pref = 1.0;
        for (int k = 0; k < dim; ++k) {
            const double ak = params[k], ck = params[dim + k];
            if (!(ck > 0.0)) return VEGAS_EINVAL;
            const double integral = ck * (std::atan(ck * (1.0 - ak)) + std::atan(ck * ak));
            pref *= ck / integral;
            fc->sc[0][k] = fc->sc[1][k] = ck;
            fc->sh[0][k] = fc->sh[1][k] = -ak * ck;
        }
        fc->C = pref * npow;
        fc->C32 = pref;
        return VEGAS_OK;
    }
    default:
        return VEGAS_EINVAL;
    }
}

// The box composed into both precisions' staging: z = sc x + sh with
// x = lo + w u becomes z = (sc w) u + (sc lo + sh); the staged widths then
// carry w, so the Jacobian gains prod w with the prefactors unchanged.
void compose_box(FnConsts* fc, int dim, const double* lo, const double* hi) {
    for (int k = 0; k < dim; ++k) {
        const double w = hi[k] - lo[k];
        for (int p = 0; p < 2; ++p) {
            fc->sh[p][k] = fc->sc[p][k] * lo[k] + fc->sh[p][k];
            fc->sc[p][k] *= w;
        }
    }
}

// Inverse-variance combination of log rows first .. n-1 (columns I = 4,
// var = 5; rows `stride` doubles apart).  An iteration with zero variance makes
// the result the plain mean with sigma 0.  NaNs when there is no row.
void combine_rows(const double* rows, int stride, int first_iter, int n, double* mean,
                  double* sigma, double* chi2_dof) {
    const int K = n - first_iter;
    double m = NAN, sg = NAN, c2 = NAN;
    if (K > 0) {
        bool zero = false;
        for (int t = first_iter; t < n; ++t)
            if (!(rows[(size_t)t * stride + 5] > 0.0)) zero = true;
        if (zero) {
            double acc = 0.0;
            for (int t = first_iter; t < n; ++t) acc += rows[(size_t)t * stride + 4];
            m = acc / K;
            sg = 0.0;
            double dev = 0.0;
            for (int t = first_iter; t < n; ++t) {
                const double d = rows[(size_t)t * stride + 4] - m;
                dev += d * d;
            }
            c2 = K > 1 ? (dev == 0.0 ? 0.0 : INFINITY) : 0.0;
        } else {
            double w = 0.0, wi = 0.0;
            for (int t = first_iter; t < n; ++t) {
                const double I = rows[(size_t)t * stride + 4];
                const double v = rows[(size_t)t * stride + 5];
                w += 1.0 / v;
                wi += I / v;
            }
            m = wi / w;
            sg = std::sqrt(1.0 / w);
            double chi = 0.0;
            for (int t = first_iter; t < n; ++t) {
                const double d = rows[(size_t)t * stride + 4] - m;
                chi += d * d / rows[(size_t)t * stride + 5];
            }
            c2 = K > 1 ? chi / (K - 1) : 0.0;
        }
    }
    *mean = m;
    *sigma = sg;
    *chi2_dof = c2;
}
}  // namespace vegas

using namespace vegas;

namespace vegas {

namespace {
// Launch shapes prepared in this process, with their device.  Entries never go
// stale (a kernel's limit only ever rises, to the device's maximum); past
// kShapeCacheEntries the oldest are overwritten.  Never destroyed: launches may
// come from other threads while the process exits.
constexpr size_t kShapeCacheEntries = 256;
struct PreparedShape {
    int device;
    const void* kern;
    int block;
    size_t smem;
    int occ;
};
struct ShapeCache {
    std::mutex mu;
    std::vector<PreparedShape> v;
    size_t next = 0;
    int optin[kMaxDevices];  // dynamic shared memory a block may take, per device (0: unknown)
};
ShapeCache& shape_cache() {
    static ShapeCache* c = new ShapeCache{};
    return *c;
}
}  // namespace

cudaError_t prepare_launch(int device, const void* kern, int block, size_t smem, int* occ) {
    if (device < 0 || device >= kMaxDevices || !kern || !occ) return cudaErrorInvalidValue;
    ShapeCache& cache = shape_cache();
    int optin = 0;
    {
        std::lock_guard<std::mutex> lock(cache.mu);
        for (const PreparedShape& c : cache.v) {
            if (c.device == device && c.kern == kern && c.block == block && c.smem == smem) {
                *occ = c.occ;
                return cudaSuccess;
            }
        }
        optin = cache.optin[device];
    }
    if (optin == 0) {
        int o = 0;
        const cudaError_t e =
            cudaDeviceGetAttribute(&o, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
        if (e != cudaSuccess) return e;
        // less what the kernels declare statically (reductions, tile index: < 1 KB)
        optin = o > 1024 ? o - 1024 : 1;
    }
    // static shared memory (~0.5 KB) counts against the 48 KB default as well;
    // the limit goes to the device's maximum, not to this shape's size, so a
    // smaller shape prepared later can never lower it under a larger one
    cudaError_t e = cudaSuccess;
    if (smem > 40 * 1024)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem > (size_t)optin ? (int)smem : optin);
    int o = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, block, smem);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(cache.mu);
        cache.optin[device] = optin;
        const PreparedShape entry{device, kern, block, smem, o};
        if (cache.v.size() < kShapeCacheEntries) cache.v.push_back(entry);
        else cache.v[cache.next++ % kShapeCacheEntries] = entry;
    }
    *occ = o;
    return cudaSuccess;
}

}  // namespace vegas

namespace {

constexpr size_t kAlign = 256;
// pinned log staging of a state: the control words, then this many log rows
constexpr int kPinnedLogRows = 4096;
constexpr size_t kPinnedCtrlBytes = 256;
static_assert(kCtrlWords * sizeof(unsigned) <= kPinnedCtrlBytes, "control words fit");

inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Log rows a state's pinned staging holds: max_iters rounded up to a power of
// two from 32, at most kPinnedLogRows, so that states of similar log lengths
// share a block size in the pool below.
int pinned_rows(int max_iters) {
    int r = 32;
    while (r < max_iters && r < kPinnedLogRows) r <<= 1;
    return r;
}

// Process-wide pool of pinned staging blocks.  Page-locking host memory costs
// the driver hundreds of microseconds per state and freeing it waits for the
// device, so vegas_destroy returns a state's block here and the next state
// that needs a block of the same size takes it; at most kPinnedPoolBlocks
// blocks wait in the pool (the rest are freed).  Every block is allocated
// portable, so any device's state may take it.
constexpr size_t kPinnedPoolBlocks = 64;
struct PinnedPool {
    std::mutex mu;
    std::vector<std::pair<void*, size_t>> free;  // (block, bytes)
};
// never destroyed: states may be released from other threads' exit paths
PinnedPool& pinned_pool() {
    static PinnedPool* pool = new PinnedPool;
    return *pool;
}

void* pinned_take(size_t bytes) {
    PinnedPool& pool = pinned_pool();
    {
        std::lock_guard<std::mutex> lock(pool.mu);
        for (size_t i = 0; i < pool.free.size(); ++i) {
            if (pool.free[i].second == bytes) {
                void* p = pool.free[i].first;
                pool.free[i] = pool.free.back();
                pool.free.pop_back();
                return p;
            }
        }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Returns the block to the pool (or frees it when the pool is full).  The
// caller has synchronised every copy that used it.
bool pinned_give(void* p, size_t bytes) {
    if (!p) return true;
    PinnedPool& pool = pinned_pool();
    {
        std::lock_guard<std::mutex> lock(pool.mu);
        if (pool.free.size() < kPinnedPoolBlocks) {
            pool.free.emplace_back(p, bytes);
            return true;
        }
    }
    return cudaFreeHost(p) == cudaSuccess;
}

struct Layout {
    size_t edges, hist, log, partials, ctrl, staged, total;
};

Layout layout(int dim, int nbins, int max_iters) {
    Layout L;
    size_t off = 0;
    L.edges = off;
    off = align_up(off + (size_t)dim * (nbins + 1) * sizeof(double));
    L.hist = off;
    off = align_up(off + (size_t)dim * nbins * sizeof(double));
    L.log = off;
    off = align_up(off + (size_t)max_iters * kLogStride * sizeof(double));
    L.partials = off;
    off = align_up(off + (size_t)kMaxGrid * kPartialStride * sizeof(double));
    L.ctrl = off;
    off = align_up(off + kCtrlWords * sizeof(unsigned));
    L.staged = off;  // float path: staged pairs of the grid
    off = align_up(off + (size_t)dim * nbins * sizeof(float2));
    L.total = off;
    return L;
}

bool shape_ok(int dim, int nbins, int max_iters) {
    return dim >= 1 && dim <= kMaxDim && nbins >= 1 && nbins <= kMaxBins &&
           dim * nbins <= kMaxDimBins && max_iters >= 1 && max_iters <= (1 << 24);
}

// Current-device guard: every call runs on the device that holds the workspace.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int cuda_status(cudaError_t e) { return e == cudaSuccess ? VEGAS_OK : VEGAS_ECUDA; }

const void* kernel_for(const vegas_state* s, bool adapt) {
    return s->mode == VEGAS_FP32_EVAL ? iterate_kernel_f32(s->integrand, s->dim, adapt)
                                      : iterate_kernel_f64(s->integrand, s->dim, adapt);
}

// Per-state cache in front of prepare_launch: a state's iterations read their
// launch shape from the descriptor, with no lock and no runtime call.
cudaError_t launch_shape(vegas_state* s, const void* kern, int block, size_t smem, int* occ) {
    for (int i = 0; i < s->n_shapes; ++i) {
        const vegas_state::LaunchShape& c = s->shapes[i];
        if (c.kern == kern && c.block == block && c.smem == smem) {
            *occ = c.occ;
            return cudaSuccess;
        }
    }
    int o = 0;
    const cudaError_t e = prepare_launch(s->device, kern, block, smem, &o);
    if (e != cudaSuccess) return e;
    constexpr int kSlots = (int)(sizeof(s->shapes) / sizeof(s->shapes[0]));
    const int slot = s->n_shapes < kSlots ? s->n_shapes++ : (s->next_shape++ % kSlots);
    s->shapes[slot] = {kern, block, smem, o};
    *occ = o;
    return cudaSuccess;
}

}  // namespace

// After any change of the grid other than a refinement (which stages its own
// result): rewrite the float path's staged pairs.  Enqueued on the stream.
int restage(vegas_state* s) {
    if (!s->staged32) return VEGAS_OK;
    return cuda_status(launch_stage32(s->edges, s->staged32, s->dim, s->nbins, s->fc, s->stream));
}

namespace {

void default_config(vegas_config* c) {
    c->block_threads = 256;
    c->blocks_per_sm = 0;
    c->min_samples_per_thread = 8;
    c->chunk_samples = 0;
}

}  // namespace

extern "C" {

int vegas_workspace_bytes(int dim, int nbins, int max_iters, size_t* bytes) {
    if (!bytes || !shape_ok(dim, nbins, max_iters)) return VEGAS_EINVAL;
    *bytes = layout(dim, nbins, max_iters).total;
    return VEGAS_OK;
}

int vegas_init_grid(vegas_state** out, int dim, int nbins, uint64_t seed, int mode, int integrand,
                    const double* params, int nparams, int max_iters, void* d_workspace,
                    size_t ws_bytes, void* cuda_stream) {
    vegas::TraceRange trace_("vegas_init_grid");
    if (!out) return VEGAS_EINVAL;
    *out = nullptr;
    if (!shape_ok(dim, nbins, max_iters) || !d_workspace) return VEGAS_EINVAL;
    if (mode != VEGAS_FP64 && mode != VEGAS_FP32_EVAL) return VEGAS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_workspace) % kAlign) != 0) return VEGAS_EINVAL;
    const Layout L = layout(dim, nbins, max_iters);
    if (ws_bytes < L.total) return VEGAS_ENOSPACE;

    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, d_workspace) != cudaSuccess ||
        attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return VEGAS_EINVAL;
    }

    vegas_state* s = new (std::nothrow) vegas_state;
    if (!s) return VEGAS_EINVAL;
    std::memset(s, 0, sizeof(*s));
    s->dim = dim;
    s->nbins = nbins;
    s->mode = mode;
    s->integrand = integrand;
    s->max_iters = max_iters;
    s->seed = seed;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->device = attr.device;
    int rc = make_consts(integrand, dim, nbins, params, nparams, &s->fc);
    if (rc != VEGAS_OK) { delete s; return rc; }
    s->nparams = !params || nparams < 0 ? 0 : (nparams > 1 + 2 * kMaxDim ? 1 + 2 * kMaxDim
                                                                           : nparams);
    for (int i = 0; i < s->nparams; ++i) s->params[i] = params[i];
    philox_round_keys(seed, s->rk0, s->rk1);
    default_config(&s->cfg);

    DeviceGuard g(s->device);
    if (!g.ok) { delete s; return VEGAS_ECUDA; }
    int optin = 0;
    if (cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device) !=
            cudaSuccess) {
        delete s;
        return VEGAS_ECUDA;
    }
    // dynamic shared memory a block may take, less what the kernels declare
    // statically (reductions and the tile index, under 1 KB)
    s->smem_optin = optin > 1024 ? optin - 1024 : 0;
    s->ws = static_cast<unsigned char*>(d_workspace);
    s->ws_bytes = ws_bytes;
    s->edges = reinterpret_cast<double*>(s->ws + L.edges);
    s->hist = reinterpret_cast<double*>(s->ws + L.hist);
    s->log = reinterpret_cast<double*>(s->ws + L.log);
    s->partials = reinterpret_cast<double*>(s->ws + L.partials);
    s->ctrl = reinterpret_cast<unsigned*>(s->ws + L.ctrl);
    s->staged32 =
        mode == VEGAS_FP32_EVAL ? reinterpret_cast<float2*>(s->ws + L.staged) : nullptr;

    // pinned staging for reading the log back: the control words and up to
    // kPinnedLogRows rows (longer logs are read through it in pieces), from
    // the pool of blocks that destroyed states returned
    s->pin_rows = pinned_rows(max_iters);
    s->pin_bytes = kPinnedCtrlBytes + (size_t)s->pin_rows * kLogStride * sizeof(double);
    void* pin = pinned_take(s->pin_bytes);
    if (!pin) {
        delete s;
        return VEGAS_ECUDA;
    }
    s->pin_ctrl = static_cast<unsigned*>(pin);
    s->pin_rows_buf = reinterpret_cast<double*>(static_cast<unsigned char*>(pin) + kPinnedCtrlBytes);

    rc = cuda_status(launch_init(s->edges, s->hist, s->log, s->ctrl, dim, nbins, max_iters,
                                 s->stream));
    if (rc == VEGAS_OK) rc = restage(s);
    if (rc != VEGAS_OK) {
        pinned_give(pin, s->pin_bytes);  // no copy into it was enqueued
        delete s;
        return rc;
    }
    *out = s;
    return VEGAS_OK;
}

int vegas_set_config(vegas_state* s, const vegas_config* cfg) {
    if (!s) return VEGAS_EINVAL;
    vegas_config c;
    default_config(&c);
    if (cfg) {
        if (cfg->block_threads) c.block_threads = cfg->block_threads;
        if (cfg->blocks_per_sm) c.blocks_per_sm = cfg->blocks_per_sm;
        if (cfg->min_samples_per_thread) c.min_samples_per_thread = cfg->min_samples_per_thread;
        c.chunk_samples = cfg->chunk_samples;
    }
    if (c.block_threads < 32 || c.block_threads > 256 || c.block_threads % 32 != 0 ||
        c.blocks_per_sm < 0 || c.blocks_per_sm > 64 || c.min_samples_per_thread < 1)
        return VEGAS_EINVAL;
    s->cfg = c;
    return VEGAS_OK;
}

// One iteration over the sample indices [begin, end): chunked launches of the
// iterate kernel; the log row gets this range's sums, n = end - begin.
static int enqueue_iteration(vegas_state* s, uint64_t begin, uint64_t end, int adapt) {
    vegas::TraceRange trace_("vegas_iterate");
    const uint64_t n_samples = end - begin;
    if (s->host_iters >= s->max_iters) return VEGAS_ESTATE;
    if (injected_failure(s)) return VEGAS_ECUDA;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;

    const bool ad = adapt != 0;
    const bool user = s->integrand == VEGAS_USER;
    if (user && !s->user.launch) return VEGAS_ESTATE;
    const void* kern = user ? nullptr : kernel_for(s, ad);  // the big-block shape may replace it
    if (!user && !kern) return VEGAS_EINVAL;
    int log2r = ad ? hist_log2r(s->mode, s->dim, s->nbins) : 0;
    int block = s->cfg.block_threads;
    const bool default_cfg = s->cfg.block_threads == 256 && s->cfg.blocks_per_sm == 0;
    // A float adapting iteration whose 32 lane-owned histogram copies miss the
    // default budget runs as one big block per SM when they fit its shared
    // memory: no two lanes of a warp then share a copy (no retried
    // compare-and-swap adds, no bank conflicts) at the same occupancy.  Only
    // under the default launch configuration.
    if (ad && !user && s->mode == VEGAS_FP32_EVAL && log2r < 5 && default_cfg &&
        iterate_smem_bytes(s->mode, s->dim, s->nbins, true, 5) <= (size_t)s->smem_optin &&
        iterate_kernel_f32_big(s->integrand, s->dim)) {
        log2r = 5;
        block = kBigBlockThreads;
        kern = iterate_kernel_f32_big(s->integrand, s->dim);
    }
    // the float adapting kernels of the default table run 32 copies; fewer
    // take the kernel with the run-time count
    if (ad && !user && s->mode == VEGAS_FP32_EVAL && log2r < 5 && block != kBigBlockThreads)
        kern = iterate_kernel_f32_few(s->integrand, s->dim);
    // fixed-grid float iterations at the compiled bin count (under the default
    // launch configuration)
    if (!ad && !user && s->mode == VEGAS_FP32_EVAL && default_cfg && s->nbins == kFixedBins &&
        iterate_kernel_f32_nb(s->integrand, s->dim))
        kern = iterate_kernel_f32_nb(s->integrand, s->dim);
    if (!user && !kern) return VEGAS_EINVAL;
    const size_t smem = iterate_smem_bytes(s->mode, s->dim, s->nbins, ad, log2r);
    int occ = 0;
    if (user) {
        // the caller's kernels: prepared on the first iteration of each kind
        // (fixed or adapting) and kept in the descriptor
        vegas_state::UserShape& us = s->user_shape[ad ? 1 : 0];
        if (us.occ < 1 || us.block != block || us.smem != smem) {
            int o = 0;
            if (s->user.prepare(s->mode, ad ? 1 : 0, block, smem, &o) != 0 || o < 1)
                return VEGAS_ECUDA;
            us = {block, smem, o};
        }
        occ = us.occ;
    } else if (launch_shape(s, kern, block, smem, &occ) != cudaSuccess || occ < 1) {
        return VEGAS_ECUDA;
    }
    const int bps = s->cfg.blocks_per_sm > 0 && s->cfg.blocks_per_sm < occ ? s->cfg.blocks_per_sm
                                                                           : occ;
    long long grid_max = (long long)s->sm_count * bps;
    if (grid_max > kMaxGrid) grid_max = kMaxGrid;

    // launches of at most 2^40 samples keep the grid-stride loop's index far
    // from overflow; the user's chunk size splits further
    uint64_t chunk = s->cfg.chunk_samples ? s->cfg.chunk_samples : n_samples;
    const uint64_t kMaxChunk = 1ull << 40;
    if (chunk > kMaxChunk) chunk = kMaxChunk;

    IterArgs a;
    std::memset(&a, 0, sizeof(a));
    a.edges = s->edges;
    a.hist = s->hist;
    a.partials = s->partials;
    a.log = s->log;
    a.ctrl = s->ctrl;
    a.n_total = n_samples;
    a.nbins = s->nbins;
    a.max_iters = s->max_iters;
    a.hist_log2r = log2r;
    a.integral_id = 0;
    std::memcpy(a.rk0, s->rk0, sizeof(a.rk0));
    std::memcpy(a.rk1, s->rk1, sizeof(a.rk1));
    a.fc = s->fc;
    a.staged32 = s->staged32;
    fill_row_offsets(s->nbins, a.rowoff);

    for (uint64_t i0 = begin; i0 < end; i0 += chunk) {
        const uint64_t nc = (end - i0) < chunk ? (end - i0) : chunk;
        a.i0 = i0;
        a.n_chunk = nc;
        a.first_chunk = i0 == begin;
        a.last_chunk = i0 + nc == end;
        const uint64_t per_block = (uint64_t)block * s->cfg.min_samples_per_thread;
        long long grid = (long long)((nc + per_block - 1) / per_block);
        if (grid > grid_max) grid = grid_max;
        if (grid < 1) grid = 1;
        if (user) {
            if (s->user.launch(s->mode, ad ? 1 : 0, &a, (unsigned)grid, (unsigned)block, smem,
                               s->stream) != 0)
                return VEGAS_ECUDA;
        } else {
            void* args[] = {&a};
            if (cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(block), args, smem, s->stream) !=
                cudaSuccess)
                return VEGAS_ECUDA;
        }
    }
    s->host_iters++;
    return VEGAS_OK;
}

int vegas_set_box(vegas_state* s, const double* lo, const double* hi) {
    if (!s) return VEGAS_EINVAL;
    if (s->host_iters != 0) return VEGAS_ESTATE;
    double w[kMaxDim];
    for (int k = 0; k < s->dim; ++k) {
        if (!lo || !hi || !std::isfinite(lo[k]) || !std::isfinite(hi[k]) || !(hi[k] > lo[k]))
            return VEGAS_EINVAL;
        w[k] = hi[k] - lo[k];
        if (!std::isfinite(w[k])) return VEGAS_EINVAL;
    }
    // the integrand's constants afresh, then the box composed into them
    FnConsts fc;
    const int rc = make_consts(s->integrand, s->dim, s->nbins, s->params, s->nparams, &fc);
    if (rc != VEGAS_OK) return rc;
    compose_box(&fc, s->dim, lo, hi);
    fc.user = s->fc.user;
    s->fc = fc;
    s->has_box = 1;
    for (int k = 0; k < s->dim; ++k) {
        s->box_lo[k] = lo[k];
        s->box_hi[k] = hi[k];
    }
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    return restage(s);
}

int vegas_inject_failure(vegas_state* s, int countdown) {
    if (!s || countdown < 0) return VEGAS_EINVAL;
    s->inject_countdown = countdown;
    return VEGAS_OK;
}

int vegas_set_user_integrand(vegas_state* s, const vegas_user_integrand* u, const void* d_data) {
    if (!s || !u || s->integrand != VEGAS_USER || u->dim != s->dim ||
        u->args_bytes != sizeof(IterArgs) || !u->prepare || !u->launch)
        return VEGAS_EINVAL;
    s->user = *u;
    s->user_shape[0] = s->user_shape[1] = {};  // new kernels: prepare them again
    s->fc.user = d_data;
    return VEGAS_OK;
}

int vegas_iterate(vegas_state* s, uint64_t n_samples, int adapt) {
    if (!s || n_samples < 2 || n_samples > VEGAS_MAX_SAMPLE_INDEX) return VEGAS_EINVAL;
    return enqueue_iteration(s, 0, n_samples, adapt);
}

int vegas_iterate_range(vegas_state* s, uint64_t n_total, uint64_t i_begin, uint64_t i_end,
                        int adapt) {
    if (!s || n_total < 2 || n_total > VEGAS_MAX_SAMPLE_INDEX || i_begin >= i_end ||
        i_end > n_total)
        return VEGAS_EINVAL;
    return enqueue_iteration(s, i_begin, i_end, adapt);
}

int vegas_shard_export(vegas_state* s, double* d_buf) {
    if (!s || !device_memory_on(d_buf, s->device)) return VEGAS_EINVAL;
    if (s->host_iters < 1) return VEGAS_ESTATE;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    const double* row = s->log + (size_t)(s->host_iters - 1) * kLogStride;
    // {S1, S2} then nonfinite (row columns 0, 1, 3), then the histogram
    if (cudaMemcpyAsync(d_buf, row, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_buf + 2, row + 3, sizeof(double), cudaMemcpyDeviceToDevice,
                        s->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_buf + 3, s->hist, (size_t)s->dim * s->nbins * sizeof(double),
                        cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
        return VEGAS_ECUDA;
    return VEGAS_OK;
}

int vegas_shard_import(vegas_state* s, const double* d_buf, uint64_t n_total) {
    if (!s || n_total < 2 || n_total > VEGAS_MAX_SAMPLE_INDEX ||
        !device_memory_on(d_buf, s->device))
        return VEGAS_EINVAL;
    if (s->host_iters < 1) return VEGAS_ESTATE;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    if (cudaMemcpyAsync(s->hist, d_buf + 3, (size_t)s->dim * s->nbins * sizeof(double),
                        cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
        return VEGAS_ECUDA;
    return cuda_status(launch_shard_rows(s->log + (size_t)(s->host_iters - 1) * kLogStride, d_buf,
                                         1, n_total, s->stream));
}

int vegas_shard_export_rows(vegas_state* s, int first_iter, int count, double* d_buf) {
    if (!s || first_iter < 0 || count < 1 || !device_memory_on(d_buf, s->device))
        return VEGAS_EINVAL;
    if (first_iter + count > s->host_iters) return VEGAS_ESTATE;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    const double* rows = s->log + (size_t)first_iter * kLogStride;
    // per row {S1, S2} (columns 0, 1) then nonfinite (column 3), 3 doubles apart
    const size_t pitch = kLogStride * sizeof(double), out = 3 * sizeof(double);
    if (cudaMemcpy2DAsync(d_buf, out, rows, pitch, 2 * sizeof(double), (size_t)count,
                          cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
        cudaMemcpy2DAsync(d_buf + 2, out, rows + 3, pitch, sizeof(double), (size_t)count,
                          cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
        return VEGAS_ECUDA;
    return VEGAS_OK;
}

int vegas_shard_import_rows(vegas_state* s, int first_iter, int count, const double* d_buf,
                            uint64_t n_total) {
    if (!s || first_iter < 0 || count < 1 || n_total < 2 || n_total > VEGAS_MAX_SAMPLE_INDEX ||
        !device_memory_on(d_buf, s->device))
        return VEGAS_EINVAL;
    if (first_iter + count > s->host_iters) return VEGAS_ESTATE;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    return cuda_status(launch_shard_rows(s->log + (size_t)first_iter * kLogStride, d_buf, count,
                                         n_total, s->stream));
}

int vegas_grid_digest(vegas_state* s, uint64_t* d_out) {
    if (!s || (reinterpret_cast<uintptr_t>(d_out) % 8) != 0 || !device_memory_on(d_out, s->device))
        return VEGAS_EINVAL;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    return cuda_status(launch_grid_digest(s->edges, s->dim * (s->nbins + 1),
                                          reinterpret_cast<unsigned long long*>(d_out), s->stream));
}

int vegas_refine(vegas_state* s, double alpha) {
    vegas::TraceRange trace_("vegas_refine");
    if (!s || !(alpha >= 0.0) || !std::isfinite(alpha)) return VEGAS_EINVAL;
    if (injected_failure(s)) return VEGAS_ECUDA;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    RefineArgs r{};
    r.edges = s->edges;
    r.hist = s->hist;
    r.dim = s->dim;
    r.nbins = s->nbins;
    r.alpha = alpha;
    r.staged32 = s->staged32;
    for (int k = 0; k < kMaxDim; ++k) {
        r.sc32[k] = s->fc.sc[1][k];
        r.sh32[k] = s->fc.sh[1][k];
    }
    return cuda_status(launch_refine(r, s->stream));
}

// The device's iteration count and the first min(count, max_rows) log rows,
// read through the state's pinned staging: one copy and one stream
// synchronisation for the control words, one each for the rows when they fit
// the staging (longer logs go through it in pieces into `heap`).  *rows points
// at the rows until the next read.
static int read_log(vegas_state* s, int max_rows, const double** rows, int* n_rows,
                    std::unique_ptr<double[]>* heap) {
    if (cudaMemcpyAsync(s->pin_ctrl, s->ctrl, kCtrlWords * sizeof(unsigned),
                        cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
        return VEGAS_ECUDA;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return VEGAS_ECUDA;
    if (s->pin_ctrl[kStatus] & (kStatusLogFull | kStatusCheckFailed)) return VEGAS_ESTATE;
    int n = (int)s->pin_ctrl[kIter];
    if (n > max_rows) n = max_rows;
    const size_t row_bytes = kLogStride * sizeof(double);
    *rows = s->pin_rows_buf;
    if (n > s->pin_rows) {
        heap->reset(new (std::nothrow) double[(size_t)n * kLogStride]);
        if (!*heap) return VEGAS_EINVAL;
        *rows = heap->get();
    }
    for (int t0 = 0; t0 < n; t0 += s->pin_rows) {
        const int m = n - t0 < s->pin_rows ? n - t0 : s->pin_rows;
        if (cudaMemcpyAsync(s->pin_rows_buf, s->log + (size_t)t0 * kLogStride, m * row_bytes,
                            cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
            return VEGAS_ECUDA;
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) return VEGAS_ECUDA;
        if (*heap) std::memcpy(heap->get() + (size_t)t0 * kLogStride, s->pin_rows_buf, m * row_bytes);
    }
    *n_rows = n;
    return VEGAS_OK;
}

static bool any_nonfinite(const double* rows, int first, int end) {
    for (int t = first; t < end; ++t)
        if (rows[(size_t)t * kLogStride + 3] != 0.0) return true;
    return false;
}

int vegas_result(vegas_state* s, int first_iter, double* mean, double* sigma, double* chi2_dof,
                 int* n_iter) {
    vegas::TraceRange trace_("vegas_result");
    if (!s || first_iter < 0) return VEGAS_EINVAL;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    const double* rows = nullptr;
    std::unique_ptr<double[]> heap;
    int n = 0;
    const int rc = read_log(s, s->max_iters, &rows, &n, &heap);
    if (rc != VEGAS_OK) return rc;
    if (n_iter) *n_iter = n;
    double m = NAN, sg = NAN, c2 = NAN;
    combine_rows(rows, kLogStride, first_iter, n, &m, &sg, &c2);
    if (mean) *mean = m;
    if (sigma) *sigma = sg;
    if (chi2_dof) *chi2_dof = c2;
    return any_nonfinite(rows, first_iter, n) ? VEGAS_ENONFINITE : VEGAS_OK;
}

int vegas_result_range(vegas_state* s, int first_iter, int end_iter, double* mean,
                       double* sigma, double* chi2_dof) {
    if (!s || first_iter < 0 || end_iter <= first_iter) return VEGAS_EINVAL;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    const double* rows = nullptr;
    std::unique_ptr<double[]> heap;
    int n = 0;
    const int rc = read_log(s, s->max_iters, &rows, &n, &heap);
    if (rc != VEGAS_OK) return rc;
    if (end_iter > n) return VEGAS_EINVAL;  // not logged (yet)
    double m = NAN, sg = NAN, c2 = NAN;
    combine_rows(rows, kLogStride, first_iter, end_iter, &m, &sg, &c2);
    if (mean) *mean = m;
    if (sigma) *sigma = sg;
    if (chi2_dof) *chi2_dof = c2;
    return any_nonfinite(rows, first_iter, end_iter) ? VEGAS_ENONFINITE : VEGAS_OK;
}

int vegas_get_iterations(vegas_state* s, double* host_rows, int max_rows, int* n_rows) {
    if (!s || !host_rows || max_rows < 0 || !n_rows) return VEGAS_EINVAL;
    *n_rows = 0;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    const double* rows = nullptr;
    std::unique_ptr<double[]> heap;
    int n = 0;
    const int rc = read_log(s, max_rows < s->max_iters ? max_rows : s->max_iters, &rows, &n, &heap);
    if (rc != VEGAS_OK) return rc;
    for (int t = 0; t < n; ++t)
        for (int c = 0; c < 6; ++c) host_rows[(size_t)t * 6 + c] = rows[(size_t)t * kLogStride + c];
    *n_rows = n;
    return VEGAS_OK;
}

int vegas_get_iteration_times(vegas_state* s, double* host_ns, int max_rows, int* n_rows) {
    if (!s || !host_ns || max_rows < 0 || !n_rows) return VEGAS_EINVAL;
    *n_rows = 0;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    const double* rows = nullptr;
    std::unique_ptr<double[]> heap;
    int n = 0;
    const int rc = read_log(s, max_rows < s->max_iters ? max_rows : s->max_iters, &rows, &n, &heap);
    if (rc != VEGAS_OK) return rc;
    for (int t = 0; t < n; ++t) host_ns[t] = rows[(size_t)t * kLogStride + 6];
    *n_rows = n;
    return VEGAS_OK;
}

int vegas_get_grid(vegas_state* s, double* host_edges) {
    if (!s || !host_edges) return VEGAS_EINVAL;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    const size_t bytes = (size_t)s->dim * (s->nbins + 1) * sizeof(double);
    if (cudaMemcpyAsync(host_edges, s->edges, bytes, cudaMemcpyDeviceToHost, s->stream) !=
        cudaSuccess)
        return VEGAS_ECUDA;
    return cuda_status(cudaStreamSynchronize(s->stream));
}

int vegas_set_grid(vegas_state* s, const double* host_edges) {
    if (!s || !host_edges) return VEGAS_EINVAL;
    const int N = s->nbins;
    for (int k = 0; k < s->dim; ++k) {
        const double* e = host_edges + (size_t)k * (N + 1);
        if (e[0] != 0.0 || e[N] != 1.0) return VEGAS_ESTATE;
        for (int l = 0; l < N; ++l)
            if (!(e[l + 1] > e[l])) return VEGAS_ESTATE;
    }
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    const size_t bytes = (size_t)s->dim * (N + 1) * sizeof(double);
    if (cudaMemcpyAsync(s->edges, host_edges, bytes, cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess)
        return VEGAS_ECUDA;
    const int rc = restage(s);
    if (rc != VEGAS_OK) return rc;
    return cuda_status(cudaStreamSynchronize(s->stream));
}

int vegas_get_histogram(vegas_state* s, double* host_hist) {
    if (!s || !host_hist) return VEGAS_EINVAL;
    DeviceGuard g(s->device);
    if (!g.ok) return VEGAS_ECUDA;
    const size_t bytes = (size_t)s->dim * s->nbins * sizeof(double);
    if (cudaMemcpyAsync(host_hist, s->hist, bytes, cudaMemcpyDeviceToHost, s->stream) !=
        cudaSuccess)
        return VEGAS_ECUDA;
    return cuda_status(cudaStreamSynchronize(s->stream));
}

int vegas_destroy(vegas_state* s) {
    if (!s) return VEGAS_OK;
    int rc = VEGAS_OK;
    {
        DeviceGuard g(s->device);
        if (g.ok && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = VEGAS_ECUDA;
        // copies into the staging are synchronised by the calls that make them
        if (!pinned_give(s->pin_ctrl, s->pin_bytes)) rc = VEGAS_ECUDA;
    }
    delete s;
    return rc;
}

const char* vegas_strerror(int status) {
    switch (status) {
    case VEGAS_OK: return "ok";
    case VEGAS_EINVAL: return "invalid argument";
    case VEGAS_ECUDA: return "CUDA runtime error";
    case VEGAS_ENONFINITE: return "non-finite integrand value (left out of the sums)";
    case VEGAS_ESTATE: return "invalid state (call order, full iteration log or bad grid)";
    case VEGAS_ENOSPACE: return "workspace too small";
    default: return "unknown status";
    }
}

}  // extern "C"
