// vegas_export_state / vegas_import_state: a state's resumable content as a
// flat little-endian blob (include/vegas.h).
//
// Layout, every field 8 bytes:
//   magic "VEGASB3" + NUL, format version (2; version 1 blobs, without the
//   box, are read too),
//   dim, nbins, mode, integrand, max_iters, nparams, seed, n_iter,
//   block_threads, blocks_per_sm, min_samples_per_thread, chunk_samples,
//   has_box, unused,
//   params[nparams], edges[dim (nbins+1)], hist[dim nbins], log[n_iter x 8],
//   and when has_box: box_lo[dim], box_hi[dim].
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "vegas_internal.h"

namespace {

constexpr char kMagic[8] = {'V', 'E', 'G', 'A', 'S', 'B', '3', 0};
constexpr uint64_t kVersion = 2;
constexpr size_t kHeaderWords = 16;

bool little_endian() {
    const uint32_t one = 1;
    unsigned char b;
    std::memcpy(&b, &one, 1);
    return b == 1;
}

size_t blob_bytes(uint64_t dim, uint64_t nbins, uint64_t nparams, uint64_t n_iter,
                  bool has_box) {
    return 8 * (kHeaderWords + nparams + dim * (nbins + 1) + dim * nbins +
                n_iter * vegas::kLogStride + (has_box ? 2 * dim : 0));
}

}  // namespace

extern "C" int vegas_export_state(vegas_state* s, void* buf, size_t* bytes) {
    using namespace vegas;
    if (!s || !bytes) return VEGAS_EINVAL;
    if (!little_endian()) return VEGAS_EINVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return VEGAS_ECUDA;
    if (prev != s->device && cudaSetDevice(s->device) != cudaSuccess) return VEGAS_ECUDA;
    int rc = VEGAS_OK;
    unsigned ctrl[kCtrlWords];
    if (cudaMemcpyAsync(ctrl, s->ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        rc = VEGAS_ECUDA;
    const uint64_t n_iter = rc == VEGAS_OK ? ctrl[kIter] : 0;
    const uint64_t dim = s->dim, nbins = s->nbins, np = s->nparams;
    const size_t need = blob_bytes(dim, nbins, np, n_iter, s->has_box != 0);
    if (rc == VEGAS_OK && !buf) {
        *bytes = need;
    } else if (rc == VEGAS_OK) {
        if (*bytes < need) {
            rc = VEGAS_ENOSPACE;
        } else {
            unsigned char* p = static_cast<unsigned char*>(buf);
            uint64_t head[kHeaderWords];
            std::memcpy(&head[0], kMagic, 8);
            head[1] = kVersion;
            head[2] = dim;
            head[3] = nbins;
            head[4] = (uint64_t)s->mode;
            head[5] = (uint64_t)s->integrand;
            head[6] = (uint64_t)s->max_iters;
            head[7] = np;
            head[8] = s->seed;
            head[9] = n_iter;
            head[10] = (uint64_t)s->cfg.block_threads;
            head[11] = (uint64_t)s->cfg.blocks_per_sm;
            head[12] = (uint64_t)s->cfg.min_samples_per_thread;
            head[13] = s->cfg.chunk_samples;
            head[14] = s->has_box ? 1 : 0;
            head[15] = 0;
            std::memcpy(p, head, sizeof(head));
            p += sizeof(head);
            std::memcpy(p, s->params, 8 * np);
            p += 8 * np;
            if (cudaMemcpyAsync(p, s->edges, 8 * dim * (nbins + 1), cudaMemcpyDeviceToHost,
                                s->stream) != cudaSuccess)
                rc = VEGAS_ECUDA;
            p += 8 * dim * (nbins + 1);
            if (rc == VEGAS_OK && cudaMemcpyAsync(p, s->hist, 8 * dim * nbins,
                                                  cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
                rc = VEGAS_ECUDA;
            p += 8 * dim * nbins;
            if (rc == VEGAS_OK && n_iter &&
                cudaMemcpyAsync(p, s->log, 8 * n_iter * kLogStride, cudaMemcpyDeviceToHost,
                                s->stream) != cudaSuccess)
                rc = VEGAS_ECUDA;
            p += 8 * n_iter * kLogStride;
            if (s->has_box) {
                std::memcpy(p, s->box_lo, 8 * dim);
                std::memcpy(p + 8 * dim, s->box_hi, 8 * dim);
            }
            if (rc == VEGAS_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = VEGAS_ECUDA;
            *bytes = need;
        }
    }
    if (prev != s->device) cudaSetDevice(prev);
    return rc;
}

extern "C" int vegas_import_state(vegas_state** out, const void* buf, size_t bytes,
                                  void* d_workspace, size_t ws_bytes, void* cuda_stream) {
    using namespace vegas;
    if (!out) return VEGAS_EINVAL;
    *out = nullptr;
    if (!buf || bytes < 8 * kHeaderWords || !little_endian()) return VEGAS_EINVAL;
    uint64_t head[kHeaderWords];
    std::memcpy(head, buf, sizeof(head));
    if (std::memcmp(&head[0], kMagic, 8) != 0 || (head[1] != 1 && head[1] != kVersion))
        return VEGAS_EINVAL;
    const bool has_box = head[1] >= 2 && head[14] != 0;
    const uint64_t dim = head[2], nbins = head[3], np = head[7], n_iter = head[9];
    const uint64_t max_iters = head[6];
    if (dim < 1 || dim > (uint64_t)kMaxDim || nbins < 1 || nbins > (uint64_t)kMaxBins ||
        np > 1 + 2 * (uint64_t)kMaxDim || max_iters < 1 || max_iters > (1u << 24) ||
        n_iter > max_iters)
        return VEGAS_EINVAL;
    if (bytes != blob_bytes(dim, nbins, np, n_iter, has_box)) return VEGAS_EINVAL;
    const unsigned char* p = static_cast<const unsigned char*>(buf) + sizeof(head);
    std::vector<double> params(np ? np : 1);
    std::memcpy(params.data(), p, 8 * np);
    p += 8 * np;
    {  // the grid must be one vegas_set_grid accepts: 0 and 1 at the ends, increasing
        std::vector<double> e(nbins + 1);
        for (uint64_t k = 0; k < dim; ++k) {
            std::memcpy(e.data(), p + 8 * k * (nbins + 1), 8 * (nbins + 1));
            if (e[0] != 0.0 || e[nbins] != 1.0) return VEGAS_EINVAL;
            for (uint64_t l = 0; l < nbins; ++l)
                if (!(e[l + 1] > e[l])) return VEGAS_EINVAL;
        }
    }
    vegas_state* s = nullptr;
    int rc = vegas_init_grid(&s, (int)dim, (int)nbins, head[8], (int)head[4], (int)head[5],
                             np ? params.data() : nullptr, (int)np, (int)max_iters, d_workspace,
                             ws_bytes, cuda_stream);
    if (rc != VEGAS_OK) return rc;
    if (has_box) {  // after the log: box_lo[dim], box_hi[dim]
        const unsigned char* b =
            p + 8 * (dim * (nbins + 1) + dim * nbins + n_iter * kLogStride);
        double lo[kMaxDim], hi[kMaxDim];
        std::memcpy(lo, b, 8 * dim);
        std::memcpy(hi, b + 8 * dim, 8 * dim);
        rc = vegas_set_box(s, lo, hi);
        if (rc != VEGAS_OK) {
            vegas_destroy(s);
            return VEGAS_EINVAL;
        }
    }
    vegas_config cfg;
    cfg.block_threads = (int)head[10];
    cfg.blocks_per_sm = (int)head[11];
    cfg.min_samples_per_thread = (int)head[12];
    cfg.chunk_samples = head[13];
    rc = vegas_set_config(s, &cfg);
    int prev = -1;
    if (rc == VEGAS_OK && cudaGetDevice(&prev) != cudaSuccess) rc = VEGAS_ECUDA;
    if (rc == VEGAS_OK && prev != s->device && cudaSetDevice(s->device) != cudaSuccess)
        rc = VEGAS_ECUDA;
    unsigned ctrl[kCtrlWords] = {};
    ctrl[kIter] = (unsigned)n_iter;
    if (rc == VEGAS_OK &&
        (cudaMemcpyAsync(s->edges, p, 8 * dim * (nbins + 1), cudaMemcpyHostToDevice,
                         s->stream) != cudaSuccess ||
         restage(s) != VEGAS_OK ||
         cudaMemcpyAsync(s->hist, p + 8 * dim * (nbins + 1), 8 * dim * nbins,
                         cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
         (n_iter && cudaMemcpyAsync(s->log, p + 8 * (dim * (nbins + 1) + dim * nbins),
                                    8 * n_iter * kLogStride, cudaMemcpyHostToDevice,
                                    s->stream) != cudaSuccess) ||
         cudaMemcpyAsync(s->ctrl, ctrl, sizeof(ctrl), cudaMemcpyHostToDevice, s->stream) !=
             cudaSuccess ||
         cudaStreamSynchronize(s->stream) != cudaSuccess))
        rc = VEGAS_ECUDA;
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    if (rc != VEGAS_OK) {
        vegas_destroy(s);
        return rc;
    }
    s->host_iters = (int)n_iter;
    *out = s;
    return VEGAS_OK;
}
