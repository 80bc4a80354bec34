// Host side of the batch API (include/vegas.h) and its two small kernels:
// batch_post_kernel refines every (integral, dimension) row and records each
// integral's estimate; batch_init_kernel resets grids, histograms and logs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "batch_kernel.cuh"
#include "philox.cuh"
#include "refine_row.cuh"
#include "stage.cuh"

namespace vegas {
namespace {

constexpr int kPostThreads = 256;
constexpr uint64_t kDefaultTile = 65536;
constexpr uint64_t kMinTile = 128;  // one sample per thread of a 128-thread block

struct BatchRow {
    int b, k;  // integral, dimension
};

struct PostArgs {
    const BatchRow* rows;
    const BatchInfo* info;
    const FnConsts* consts;
    float2* staged32;  // float path: staged pairs of every row (hist layout), else null
    double* edges;
    double* hist;
    double* hist_last;  // every row's histogram as the last refinement used it
    double* acc;
    double* log;
    unsigned* ctrl;
    int nbins, max_iters;
    unsigned iter;
    int adapt;
    double alpha;
};

// Block r: dimension rows[r].k of integral rows[r].b.  Adapting iterations
// keep a copy of the row's histogram (vegas_batch_get_histogram), then refine
// the row (and clear its histogram); the block of dimension 0 records
// the integral's estimate I = S1/n, var = (S2/n - I^2)/(n-1) in its log row
// `iter` and clears the accumulators; block 0 resets the tile ticket.
__global__ void __launch_bounds__(kPostThreads) batch_post_kernel(const PostArgs a) {
    extern __shared__ double sm[];
    __shared__ double sbuf[33];
    const BatchRow row = a.rows[blockIdx.x];
    const BatchInfo info = a.info[row.b];
    const int N = a.nbins;
    if (a.adapt) {
        double* e = a.edges + info.edge_off + (size_t)row.k * (N + 1);
        const size_t h0 = info.hist_off + (size_t)row.k * N;
        for (int j = threadIdx.x; j < N; j += blockDim.x) a.hist_last[h0 + j] = a.hist[h0 + j];
        __syncthreads();
        refine_row(e, a.hist + h0, N, a.alpha, sm, sbuf);
        if (a.staged32) {  // the float path's pairs of the new grid row
            __syncthreads();
            const FnConsts& fc = a.consts[row.b];
            stage_row32(e, N, fc.sc[1][row.k], fc.sh[1][row.k],
                        a.staged32 + info.hist_off + (size_t)row.k * N);
        }
    }
    if (row.k == 0 && threadIdx.x == 0) {
        double* acc = a.acc + 4 * (size_t)row.b;
        double* L = a.log + ((size_t)row.b * a.max_iters + a.iter) * kLogStride;
        const double n = (double)info.n;
        const double I = acc[0] / n;
        const double var = (acc[1] / n - I * I) / (n - 1.0);
        L[0] = acc[0];
        L[1] = acc[1];
        L[2] = n;
        L[3] = acc[2];
        L[4] = I;
        L[5] = var > 0.0 ? var : 0.0;
        L[6] = L[7] = 0.0;
        acc[0] = acc[1] = acc[2] = acc[3] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctrl[kTicket] = 0u;
        a.ctrl[kIter] = a.iter + 1;
    }
}

// Uniform grids e_l = l/N for every row, cleared histograms, accumulators,
// logs and control words.
__global__ void batch_init_kernel(double* edges, size_t n_edges, double* hist, size_t n_hist,
                                  double* hist_last, double* acc, size_t n_acc, double* log,
                                  size_t n_log, unsigned* ctrl, int nbins) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    for (size_t i = tid; i < n_edges; i += nth) edges[i] = (double)(i % (nbins + 1)) / nbins;
    for (size_t i = tid; i < n_hist; i += nth) hist[i] = hist_last[i] = 0.0;
    for (size_t i = tid; i < n_acc; i += nth) acc[i] = 0.0;
    for (size_t i = tid; i < n_log; i += nth) log[i] = 0.0;
    for (size_t i = tid; i < (size_t)kCtrlWords; i += nth) ctrl[i] = 0u;
}

// The float path's staged pairs of every (integral, dimension) row, block r
// taking row r (after the grids are reset).
__global__ void batch_stage_kernel(const BatchRow* rows, const BatchInfo* info,
                                   const FnConsts* consts, const double* edges, float2* staged,
                                   int nbins) {
    const BatchRow row = rows[blockIdx.x];
    const BatchInfo in = info[row.b];
    const FnConsts& fc = consts[row.b];
    stage_row32(edges + in.edge_off + (size_t)row.k * (nbins + 1), nbins, fc.sc[1][row.k],
                fc.sh[1][row.k], staged + in.hist_off + (size_t)row.k * nbins);
}

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct BatchLayout {
    size_t edges, hist, hist_last, acc, log, consts, info, rows, tiles, ctrl, staged, total;
    size_t n_edges, n_hist, n_rows, max_tiles;
};

bool batch_shape_ok(int count, const int* dims, const uint64_t* n, int nbins, int max_iters) {
    if (count < 1 || count > (1 << 20) || !dims || !n || nbins < 1 || nbins > kMaxBins ||
        max_iters < 1 || max_iters > (1 << 16))
        return false;
    for (int b = 0; b < count; ++b) {
        if (dims[b] < 1 || dims[b] > kMaxDim || dims[b] * nbins > kMaxDimBins) return false;
        if (n[b] < 2 || n[b] > (1ull << 40)) return false;
    }
    return true;
}

BatchLayout batch_layout(int count, const int* dims, const uint64_t* n, int nbins,
                         int max_iters) {
    BatchLayout L;
    L.n_edges = L.n_hist = L.n_rows = L.max_tiles = 0;
    for (int b = 0; b < count; ++b) {
        L.n_edges += (size_t)dims[b] * (nbins + 1);
        L.n_hist += (size_t)dims[b] * nbins;
        L.n_rows += dims[b];
        L.max_tiles += (n[b] + kMinTile - 1) / kMinTile;
    }
    size_t off = 0;
    L.edges = off; off = align_up(off + L.n_edges * sizeof(double));
    L.hist = off;  off = align_up(off + L.n_hist * sizeof(double));
    L.hist_last = off; off = align_up(off + L.n_hist * sizeof(double));
    L.acc = off;   off = align_up(off + (size_t)count * 4 * sizeof(double));
    L.log = off;   off = align_up(off + (size_t)count * max_iters * kLogStride * sizeof(double));
    L.consts = off; off = align_up(off + (size_t)count * sizeof(FnConsts));
    L.info = off;  off = align_up(off + (size_t)count * sizeof(BatchInfo));
    L.rows = off;  off = align_up(off + L.n_rows * sizeof(BatchRow));
    L.tiles = off; off = align_up(off + L.max_tiles * sizeof(BatchTile));
    L.ctrl = off;  off = align_up(off + kCtrlWords * sizeof(unsigned));
    L.staged = off; off = align_up(off + L.n_hist * sizeof(float2));
    L.total = off;
    return L;
}

}  // namespace
}  // namespace vegas

using namespace vegas;

struct vegas_batch {
    int count, nbins, mode, integrand, max_iters;
    uint64_t seed;
    cudaStream_t stream;
    int device, sm_count;
    int smem_optin;  // dynamic shared memory one block may use on this device
    unsigned char* ws;
    BatchLayout L;
    int max_dim;
    int block_threads;
    uint64_t tile_samples;
    uint64_t tile_by_dim[kMaxDim + 1];  // per dimension; 0: tile_samples
    unsigned num_tiles;
    int iters;  // iterations enqueued since the last reset
    uint32_t rk0[10], rk1[10];
    std::vector<int> dims;
    std::vector<uint64_t> n;
    std::vector<FnConsts> consts;
    std::vector<BatchInfo> info;
    std::vector<BatchRow> rows;
    std::vector<BatchTile> tiles;
};

namespace {

// Parameters of one integral of dimension d for a built-in integrand (the
// layouts of include/vegas.h).
int batch_nparams(int integrand, int d) {
    switch (integrand) {
    case VEGAS_GAUSS: return 1 + d;
    case VEGAS_GAUSS_MIX2: return 1 + 2 * d;
    case VEGAS_GENZ_DISC:
    case VEGAS_GENZ_PPEAK: return 2 * d;
    default: return 0;
    }
}

struct Dev {
    int prev = -1;
    bool ok = true;
    explicit Dev(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~Dev() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
T* at(const vegas_batch* b, size_t off) {
    return reinterpret_cast<T*>(b->ws + off);
}

// Cut every integral's samples into tiles of b->tile_samples (the last one
// shorter) and copy the table to the device.  Blocks take tiles in table
// order, so the table runs from the costliest tiles (samples x dimension) to
// the cheapest: the last tiles of an iteration, which decide how long the
// other blocks wait, are then the short ones.
int build_tiles(vegas_batch* b) {
    b->tiles.clear();
    for (int i = 0; i < b->count; ++i) {
        const uint64_t ts = b->tile_by_dim[b->dims[i]] ? b->tile_by_dim[b->dims[i]]
                                                       : b->tile_samples;
        for (uint64_t s = 0; s < b->n[i]; s += ts) {
            BatchTile t;
            t.b = (unsigned)i;
            t.start = s;
            t.count = (unsigned)((b->n[i] - s) < ts ? (b->n[i] - s) : ts);
            b->tiles.push_back(t);
        }
    }
    std::stable_sort(b->tiles.begin(), b->tiles.end(), [b](const BatchTile& x, const BatchTile& y) {
        return (uint64_t)x.count * b->dims[x.b] > (uint64_t)y.count * b->dims[y.b];
    });
    if (b->tiles.size() > b->L.max_tiles) return VEGAS_EINVAL;
    b->num_tiles = (unsigned)b->tiles.size();
    return cudaMemcpyAsync(at<BatchTile>(b, b->L.tiles), b->tiles.data(),
                           b->tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice,
                           b->stream) == cudaSuccess
               ? VEGAS_OK
               : VEGAS_ECUDA;
}

int launch_batch_init(vegas_batch* b) {
    const BatchLayout& L = b->L;
    const cudaError_t e = launch_kernel(
        batch_init_kernel, dim3(64), dim3(256), 0, b->stream, at<double>(b, L.edges), L.n_edges,
        at<double>(b, L.hist), L.n_hist, at<double>(b, L.hist_last), at<double>(b, L.acc),
        (size_t)b->count * 4,
        at<double>(b, L.log), (size_t)b->count * b->max_iters * kLogStride,
        at<unsigned>(b, L.ctrl), b->nbins);
    b->iters = 0;
    if (e != cudaSuccess) return VEGAS_ECUDA;
    if (b->mode == VEGAS_FP32_EVAL &&
        launch_kernel(batch_stage_kernel, dim3((unsigned)L.n_rows), dim3(64), 0, b->stream,
                      (const BatchRow*)at<BatchRow>(b, L.rows),
                      (const BatchInfo*)at<BatchInfo>(b, L.info),
                      (const FnConsts*)at<FnConsts>(b, L.consts), (const double*)at<double>(b, L.edges),
                      at<float2>(b, L.staged), b->nbins) != cudaSuccess)
        return VEGAS_ECUDA;
    return VEGAS_OK;
}

}  // namespace

extern "C" {

int vegas_batch_workspace_bytes(int count, const int* dims, const uint64_t* n_samples,
                                int nbins, int max_iters, size_t* bytes) {
    if (!bytes || !batch_shape_ok(count, dims, n_samples, nbins, max_iters)) return VEGAS_EINVAL;
    *bytes = batch_layout(count, dims, n_samples, nbins, max_iters).total;
    return VEGAS_OK;
}

int vegas_batch_init_integrand(vegas_batch** out, int count, const int* dims,
                               const uint64_t* n_samples, int nbins, uint64_t seed, int mode,
                               int integrand, const double* params, const double* box_lo,
                               const double* box_hi, int max_iters, void* d_workspace,
                               size_t ws_bytes, void* cuda_stream) {
    if (!out) return VEGAS_EINVAL;
    *out = nullptr;
    if (!batch_shape_ok(count, dims, n_samples, nbins, max_iters) || !d_workspace)
        return VEGAS_EINVAL;
    if (mode != VEGAS_FP64 && mode != VEGAS_FP32_EVAL) return VEGAS_EINVAL;
    if (!batch_iterate_kernel_f64(integrand, false, 256)) return VEGAS_EINVAL;  // built-in only
    if ((box_lo == nullptr) != (box_hi == nullptr)) return VEGAS_EINVAL;
    size_t total_params = 0, total_dims = 0;
    for (int i = 0; i < count; ++i) {
        total_params += batch_nparams(integrand, dims[i]);
        total_dims += dims[i];
    }
    if (total_params > 0 && !params) return VEGAS_EINVAL;
    if (box_lo)
        for (size_t k = 0; k < total_dims; ++k)
            if (!std::isfinite(box_lo[k]) || !std::isfinite(box_hi[k]) ||
                !(box_hi[k] > box_lo[k]) || !std::isfinite(box_hi[k] - box_lo[k]))
                return VEGAS_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) return VEGAS_EINVAL;
    const BatchLayout L = batch_layout(count, dims, n_samples, nbins, max_iters);
    if (ws_bytes < L.total) return VEGAS_ENOSPACE;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, d_workspace) != cudaSuccess ||
        attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return VEGAS_EINVAL;
    }
    vegas_batch* b = new (std::nothrow) vegas_batch;
    if (!b) return VEGAS_EINVAL;
    b->count = count;
    b->nbins = nbins;
    b->mode = mode;
    b->integrand = integrand;
    b->max_iters = max_iters;
    b->seed = seed;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->device = attr.device;
    b->ws = static_cast<unsigned char*>(d_workspace);
    b->L = L;
    b->block_threads = 256;
    b->tile_samples = kDefaultTile;
    for (int d = 0; d <= kMaxDim; ++d) b->tile_by_dim[d] = 0;
    b->iters = 0;
    philox_round_keys(seed, b->rk0, b->rk1);
    b->dims.assign(dims, dims + count);
    b->n.assign(n_samples, n_samples + count);
    b->consts.resize(count);
    b->info.resize(count);
    b->max_dim = 0;
    size_t eoff = 0, hoff = 0, p = 0, boff = 0;
    for (int i = 0; i < count; ++i) {
        const int np = batch_nparams(integrand, dims[i]);
        if (make_consts(integrand, dims[i], nbins, np ? params + p : nullptr, np,
                        &b->consts[i]) != VEGAS_OK) {
            delete b;
            return VEGAS_EINVAL;
        }
        if (box_lo) compose_box(&b->consts[i], dims[i], box_lo + boff, box_hi + boff);
        p += np;
        boff += dims[i];
        b->info[i].dim = dims[i];
        b->info[i].pad = 0;
        b->info[i].n = n_samples[i];
        b->info[i].edge_off = eoff;
        b->info[i].hist_off = hoff;
        eoff += (size_t)dims[i] * (nbins + 1);
        hoff += (size_t)dims[i] * nbins;
        for (int k = 0; k < dims[i]; ++k) b->rows.push_back(BatchRow{i, k});
        if (dims[i] > b->max_dim) b->max_dim = dims[i];
    }
    Dev g(b->device);
    int rc = g.ok ? VEGAS_OK : VEGAS_ECUDA;
    int optin = 0;
    if (rc == VEGAS_OK &&
        (cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device) !=
             cudaSuccess ||
         cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) !=
             cudaSuccess))
        rc = VEGAS_ECUDA;
    b->smem_optin = optin > 1024 ? optin - 1024 : 0;  // less the kernels' static shared
    if (rc == VEGAS_OK &&
        (cudaMemcpyAsync(at<FnConsts>(b, L.consts), b->consts.data(), count * sizeof(FnConsts),
                         cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
         cudaMemcpyAsync(at<BatchInfo>(b, L.info), b->info.data(), count * sizeof(BatchInfo),
                         cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
         cudaMemcpyAsync(at<BatchRow>(b, L.rows), b->rows.data(),
                         b->rows.size() * sizeof(BatchRow), cudaMemcpyHostToDevice,
                         b->stream) != cudaSuccess))
        rc = VEGAS_ECUDA;
    if (rc == VEGAS_OK) rc = build_tiles(b);
    if (rc == VEGAS_OK) rc = launch_batch_init(b);
    // the host tables above are pageable: wait for their copies before returning
    if (rc == VEGAS_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = VEGAS_ECUDA;
    if (rc != VEGAS_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return VEGAS_OK;
}

int vegas_batch_init(vegas_batch** out, int count, const int* dims, const uint64_t* n_samples,
                     int nbins, uint64_t seed, int mode, const double* params, int max_iters,
                     void* d_workspace, size_t ws_bytes, void* cuda_stream) {
    if (!params) return VEGAS_EINVAL;
    return vegas_batch_init_integrand(out, count, dims, n_samples, nbins, seed, mode,
                                      VEGAS_GAUSS, params, nullptr, nullptr, max_iters,
                                      d_workspace, ws_bytes, cuda_stream);
}

int vegas_batch_set_config(vegas_batch* b, int block_threads, uint64_t tile_samples) {
    if (!b) return VEGAS_EINVAL;
    if (block_threads && (block_threads < 32 || block_threads > 512 || block_threads % 32))
        return VEGAS_EINVAL;
    if (tile_samples && (tile_samples < kMinTile || tile_samples % 32 ||
                         tile_samples > (1ull << 31)))
        return VEGAS_EINVAL;
    if (block_threads) b->block_threads = block_threads;
    if (tile_samples && tile_samples != b->tile_samples) {
        b->tile_samples = tile_samples;
        Dev g(b->device);
        if (!g.ok) return VEGAS_ECUDA;
        const int rc = build_tiles(b);
        if (rc != VEGAS_OK) return rc;
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return VEGAS_ECUDA;
    }
    return VEGAS_OK;
}

int vegas_batch_set_tiles_by_dim(vegas_batch* b, const uint64_t* tiles, int count) {
    if (!b || count < 0 || count > kMaxDim || (count > 0 && !tiles)) return VEGAS_EINVAL;
    for (int d = 0; d < count; ++d)
        if (tiles[d] && (tiles[d] < kMinTile || tiles[d] % 32 || tiles[d] > (1ull << 31)))
            return VEGAS_EINVAL;
    for (int d = 1; d <= kMaxDim; ++d) b->tile_by_dim[d] = d <= count ? tiles[d - 1] : 0;
    Dev g(b->device);
    if (!g.ok) return VEGAS_ECUDA;
    const int rc = build_tiles(b);
    if (rc != VEGAS_OK) return rc;
    return cudaStreamSynchronize(b->stream) == cudaSuccess ? VEGAS_OK : VEGAS_ECUDA;
}

int vegas_batch_set_stream(vegas_batch* b, void* cuda_stream) {
    if (!b) return VEGAS_EINVAL;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    return VEGAS_OK;
}

int vegas_batch_reset(vegas_batch* b) {
    if (!b) return VEGAS_EINVAL;
    Dev g(b->device);
    if (!g.ok) return VEGAS_ECUDA;
    return launch_batch_init(b);
}

int vegas_batch_iterate(vegas_batch* b, int adapt, double alpha) {
    vegas::TraceRange trace_("vegas_batch_iterate");
    if (!b) return VEGAS_EINVAL;
    if (adapt && !(alpha >= 0.0 && std::isfinite(alpha))) return VEGAS_EINVAL;
    if (b->iters >= b->max_iters) return VEGAS_ESTATE;
    Dev g(b->device);
    if (!g.ok) return VEGAS_ECUDA;
    const bool ad = adapt != 0;
    const BatchLayout& L = b->L;

    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.tiles = at<BatchTile>(b, L.tiles);
    a.info = at<BatchInfo>(b, L.info);
    a.consts = at<FnConsts>(b, L.consts);
    a.edges = at<double>(b, L.edges);
    a.hist = at<double>(b, L.hist);
    a.acc = at<double>(b, L.acc);
    a.ctrl = at<unsigned>(b, L.ctrl);
    a.num_tiles = b->num_tiles;
    a.iter = (unsigned)b->iters;
    a.nbins = b->nbins;
    a.max_dim = b->max_dim;
    a.hist_log2r = ad ? hist_log2r(b->mode, b->max_dim, b->nbins) : 0;
    a.staged32 = b->mode == VEGAS_FP32_EVAL ? at<float2>(b, L.staged) : nullptr;
    std::memcpy(a.rk0, b->rk0, sizeof(a.rk0));
    std::memcpy(a.rk1, b->rk1, sizeof(a.rk1));
    fill_row_offsets(b->nbins, a.rowoff);

    int block = b->block_threads;
    const void* kern = b->mode == VEGAS_FP32_EVAL
                           ? batch_iterate_kernel_f32(b->integrand, ad, block)
                           : batch_iterate_kernel_f64(b->integrand, ad, block);
    // float adapting rounds whose 32 copies for the widest integral miss the
    // default budget run as one big block per SM when they fit it (as the
    // single-integral kernels do), at the default block size only
    if (ad && b->mode == VEGAS_FP32_EVAL && a.hist_log2r < 5 && block == 256 &&
        iterate_smem_bytes(b->mode, b->max_dim, b->nbins, true, 5) <= (size_t)b->smem_optin &&
        batch_iterate_kernel_f32_big(b->integrand)) {
        a.hist_log2r = 5;
        block = kBigBlockThreads;
        kern = batch_iterate_kernel_f32_big(b->integrand);
    }
    const size_t smem = iterate_smem_bytes(b->mode, b->max_dim, b->nbins, ad, a.hist_log2r);
    int occ = 0;
    if (prepare_launch(b->device, kern, block, smem, &occ) != cudaSuccess || occ < 1)
        return VEGAS_ECUDA;
    long long grid = (long long)b->sm_count * occ;
    if (grid > (long long)b->num_tiles) grid = b->num_tiles;
    void* args[] = {&a};
    if (cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(block), args, smem,
                         b->stream) != cudaSuccess)
        return VEGAS_ECUDA;

    PostArgs pa;
    pa.rows = at<BatchRow>(b, L.rows);
    pa.info = a.info;
    pa.consts = a.consts;
    pa.staged32 = a.staged32 ? at<float2>(b, L.staged) : nullptr;
    pa.edges = a.edges;
    pa.hist = a.hist;
    pa.hist_last = at<double>(b, L.hist_last);
    pa.acc = a.acc;
    pa.log = at<double>(b, L.log);
    pa.ctrl = a.ctrl;
    pa.nbins = b->nbins;
    pa.max_iters = b->max_iters;
    pa.iter = (unsigned)b->iters;
    pa.adapt = ad ? 1 : 0;
    pa.alpha = alpha;
    if (launch_kernel(batch_post_kernel, dim3((unsigned)L.n_rows),
                      dim3(refine_threads(b->nbins, kPostThreads)),
                      (size_t)(4 * b->nbins + 2) * sizeof(double), b->stream, pa) !=
        cudaSuccess)
        return VEGAS_ECUDA;
    b->iters++;
    return VEGAS_OK;
}

static int batch_rows(vegas_batch* b, std::vector<double>& rows, int* done) {
    unsigned ctrl[kCtrlWords];
    rows.resize((size_t)b->count * b->max_iters * kLogStride);
    if (cudaMemcpyAsync(ctrl, at<unsigned>(b, b->L.ctrl), sizeof(ctrl), cudaMemcpyDeviceToHost,
                        b->stream) != cudaSuccess ||
        cudaMemcpyAsync(rows.data(), at<double>(b, b->L.log), rows.size() * sizeof(double),
                        cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return VEGAS_ECUDA;
    if (ctrl[kStatus] & kStatusCheckFailed) return VEGAS_ESTATE;
    *done = (int)ctrl[kIter];
    return VEGAS_OK;
}

int vegas_batch_result(vegas_batch* b, int index, int first_iter, double* mean, double* sigma,
                       double* chi2_dof, int* n_iter) {
    if (!b || index < 0 || index >= b->count || first_iter < 0) return VEGAS_EINVAL;
    Dev g(b->device);
    if (!g.ok) return VEGAS_ECUDA;
    std::vector<double> rows;
    int done = 0;
    const int rc = batch_rows(b, rows, &done);
    if (rc != VEGAS_OK) return rc;
    const double* r = rows.data() + (size_t)index * b->max_iters * kLogStride;
    double m, s, c;
    combine_rows(r, kLogStride, first_iter, done, &m, &s, &c);
    int bad = 0;
    for (int t = first_iter; t < done; ++t)
        if (r[(size_t)t * kLogStride + 3] != 0.0) bad = 1;
    if (mean) *mean = m;
    if (sigma) *sigma = s;
    if (chi2_dof) *chi2_dof = c;
    if (n_iter) *n_iter = done;
    return bad ? VEGAS_ENONFINITE : VEGAS_OK;
}

int vegas_batch_get_log(vegas_batch* b, double* host_rows) {
    if (!b || !host_rows) return VEGAS_EINVAL;
    Dev g(b->device);
    if (!g.ok) return VEGAS_ECUDA;
    std::vector<double> rows;
    int done = 0;
    const int rc = batch_rows(b, rows, &done);
    if (rc != VEGAS_OK) return rc;
    for (size_t r = 0; r < (size_t)b->count * b->max_iters; ++r)
        for (int c = 0; c < 6; ++c) host_rows[r * 6 + c] = rows[r * kLogStride + c];
    return VEGAS_OK;
}

int vegas_batch_get_grid(vegas_batch* b, int index, double* host_edges) {
    if (!b || !host_edges || index < 0 || index >= b->count) return VEGAS_EINVAL;
    Dev g(b->device);
    if (!g.ok) return VEGAS_ECUDA;
    const size_t n = (size_t)b->dims[index] * (b->nbins + 1);
    if (cudaMemcpyAsync(host_edges, at<double>(b, b->L.edges) + b->info[index].edge_off,
                        n * sizeof(double), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return VEGAS_ECUDA;
    return VEGAS_OK;
}

int vegas_batch_get_histogram(vegas_batch* b, int index, double* host_hist) {
    if (!b || !host_hist || index < 0 || index >= b->count) return VEGAS_EINVAL;
    Dev g(b->device);
    if (!g.ok) return VEGAS_ECUDA;
    const size_t n = (size_t)b->dims[index] * b->nbins;
    if (cudaMemcpyAsync(host_hist, at<double>(b, b->L.hist_last) + b->info[index].hist_off,
                        n * sizeof(double), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return VEGAS_ECUDA;
    return VEGAS_OK;
}

int vegas_batch_destroy(vegas_batch* b) {
    if (!b) return VEGAS_OK;
    int rc = VEGAS_OK;
    {
        Dev g(b->device);
        if (g.ok && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = VEGAS_ECUDA;
    }
    delete b;
    return rc;
}

}  // extern "C"
