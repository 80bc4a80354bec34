"""Thin Python binding of the C ABI in include/vegas.h (ctypes).

Argument marshalling only: every step of the Vegas iteration runs in the CUDA
library ``_build/libvegas_b300.so``.  The functions keep the C names.  If the
library is missing, the first call raises -- there is no CPU fallback.
"""
import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# the library this binding loads: the release build, or another build of the
# same sources (e.g. the debug build) named by VEGAS_B300_LIBRARY
LIB_PATH = os.environ.get("VEGAS_B300_LIBRARY") or os.path.join(HERE, "_build", "libvegas_b300.so")

VEGAS_OK, VEGAS_EINVAL, VEGAS_ECUDA, VEGAS_ENONFINITE, VEGAS_ESTATE, VEGAS_ENOSPACE = range(6)
VEGAS_FP64, VEGAS_FP32_EVAL = 0, 1
VEGAS_GAUSS, VEGAS_GAUSS_MIX2, VEGAS_FLAT, VEGAS_GENZ_DISC, VEGAS_GENZ_PPEAK, VEGAS_USER = range(6)
VEGAS_MAX_DIM, VEGAS_MAX_BINS, VEGAS_MAX_DIM_X_BINS = 20, 1024, 8192
VEGAS_MAX_DEVICES = 64
VEGAS_MAX_SAMPLE_INDEX = 2**64 - 2**33
VEGAS_NOALLOC_MAX_DIM_X_BINS, VEGAS_NOALLOC_MAX_BLOCKS = 4096, 2048
LOG_COLUMNS = ("S1", "S2", "n", "nonfinite", "I", "var")
# vegas_pipe_peak operations, in the order of their VEGAS_PIPE_* codes
PIPES = ("ffma", "dfma", "ex2", "product", "imad", "lds", "atoms_u32", "atoms_f32")
VEGAS_PIPE_SCRATCH_BYTES = 64

# every symbol include/vegas.h declares
EXPORTED = ("vegas_workspace_bytes", "vegas_init_grid", "vegas_set_config", "vegas_iterate",
            "vegas_refine", "vegas_result", "vegas_get_iterations", "vegas_get_grid",
            "vegas_set_grid", "vegas_get_histogram", "vegas_sample_words", "vegas_destroy",
            "vegas_strerror", "vegas_iterate_noalloc", "vegas_gauss_adjoint",
            "vegas_batch_workspace_bytes", "vegas_batch_init", "vegas_batch_set_config",
            "vegas_batch_set_stream", "vegas_batch_reset", "vegas_batch_iterate",
            "vegas_batch_result", "vegas_batch_get_log", "vegas_batch_get_grid",
            "vegas_batch_get_histogram",
            "vegas_batch_destroy", "vegas_iterate_range", "vegas_shard_export",
            "vegas_shard_import", "vegas_export_state", "vegas_import_state",
            "vegas_set_user_integrand", "vegas_get_iteration_times",
            "vegas_batch_set_tiles_by_dim", "vegas_set_box", "vegas_pipe_peak",
            "vegas_inject_failure", "vegas_batch_init_integrand", "vegas_result_range",
            "vegas_grid_digest", "vegas_shard_export_rows", "vegas_shard_import_rows")


class VegasError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {vegas_strerror(status)} (status {status})")


class vegas_config(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("min_samples_per_thread", ctypes.c_int), ("chunk_samples", ctypes.c_uint64)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run "
                               "`python -m paper_2002_12921_b300.build`)")
        L = ctypes.CDLL(LIB_PATH)
        i32, u64, vp, dbl, sz = (ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_double,
                                 ctypes.c_size_t)
        ip = ctypes.POINTER(ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        L.vegas_workspace_bytes.argtypes = [i32, i32, i32, ctypes.POINTER(sz)]
        L.vegas_init_grid.argtypes = [ctypes.POINTER(vp), i32, i32, u64, i32, i32, vp, i32, i32,
                                      vp, sz, vp]
        L.vegas_set_config.argtypes = [vp, ctypes.POINTER(vegas_config)]
        L.vegas_set_box.argtypes = [vp, vp, vp]
        L.vegas_inject_failure.argtypes = [vp, i32]
        L.vegas_result_range.argtypes = [vp, i32, i32, vp, vp, vp]
        L.vegas_pipe_peak.argtypes = [ctypes.c_int, ctypes.c_uint32, vp, ctypes.c_size_t, vp,
                                      vp]
        L.vegas_iterate.argtypes = [vp, u64, i32]
        L.vegas_refine.argtypes = [vp, dbl]
        L.vegas_result.argtypes = [vp, i32, dp, dp, dp, ip]
        L.vegas_get_iterations.argtypes = [vp, vp, i32, ip]
        L.vegas_get_iteration_times.argtypes = [vp, vp, i32, ip]
        L.vegas_get_grid.argtypes = [vp, vp]
        L.vegas_set_grid.argtypes = [vp, vp]
        L.vegas_get_histogram.argtypes = [vp, vp]
        L.vegas_sample_words.argtypes = [u64, ctypes.c_uint32, ctypes.c_uint32, u64, u64, i32, vp,
                                         vp]
        L.vegas_iterate_noalloc.argtypes = [vp, i32, i32, u64, ctypes.c_uint32, i32, vp, i32, u64,
                                             i32, dbl, vp, vp]
        L.vegas_gauss_adjoint.argtypes = [vp, vp, i32, ctypes.c_uint32, u64, i32, vp]
        L.vegas_batch_workspace_bytes.argtypes = [i32, vp, vp, i32, i32, ctypes.POINTER(sz)]
        L.vegas_batch_init.argtypes = [ctypes.POINTER(vp), i32, vp, vp, i32, u64, i32, vp, i32,
                                       vp, sz, vp]
        L.vegas_batch_init_integrand.argtypes = [ctypes.POINTER(vp), i32, vp, vp, i32, u64, i32,
                                                 i32, vp, vp, vp, i32, vp, sz, vp]
        L.vegas_batch_set_config.argtypes = [vp, i32, u64]
        L.vegas_batch_set_tiles_by_dim.argtypes = [vp, vp, i32]
        L.vegas_batch_set_stream.argtypes = [vp, vp]
        L.vegas_batch_reset.argtypes = [vp]
        L.vegas_batch_iterate.argtypes = [vp, i32, dbl]
        L.vegas_batch_result.argtypes = [vp, i32, i32, dp, dp, dp, ip]
        L.vegas_batch_get_log.argtypes = [vp, vp]
        L.vegas_batch_get_grid.argtypes = [vp, i32, vp]
        L.vegas_batch_get_histogram.argtypes = [vp, i32, vp]
        L.vegas_batch_destroy.argtypes = [vp]
        L.vegas_iterate_range.argtypes = [vp, u64, u64, u64, i32]
        L.vegas_shard_export.argtypes = [vp, vp]
        L.vegas_shard_import.argtypes = [vp, vp, u64]
        L.vegas_shard_export_rows.argtypes = [vp, i32, i32, vp]
        L.vegas_shard_import_rows.argtypes = [vp, i32, i32, vp, u64]
        L.vegas_grid_digest.argtypes = [vp, vp]
        L.vegas_export_state.argtypes = [vp, vp, ctypes.POINTER(sz)]
        L.vegas_import_state.argtypes = [ctypes.POINTER(vp), vp, sz, vp, sz, vp]
        L.vegas_set_user_integrand.argtypes = [vp, vp, vp]
        L.vegas_destroy.argtypes = [vp]
        L.vegas_strerror.argtypes = [i32]
        L.vegas_strerror.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name != "vegas_strerror":
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(rc, where):
    if rc != VEGAS_OK:
        raise VegasError(rc, where)


def vegas_strerror(status):
    return lib().vegas_strerror(int(status)).decode()


def vegas_workspace_bytes(dim, nbins, max_iters):
    out = ctypes.c_size_t(0)
    _check(lib().vegas_workspace_bytes(dim, nbins, max_iters, ctypes.byref(out)),
           "vegas_workspace_bytes")
    return out.value


def vegas_init_grid(dim, nbins, seed, mode, integrand, params, max_iters, d_workspace, ws_bytes,
                    cuda_stream):
    """Returns the opaque handle (an int)."""
    p = np.ascontiguousarray(params if params is not None else [], dtype=np.float64)
    h = ctypes.c_void_p(None)
    _check(lib().vegas_init_grid(ctypes.byref(h), dim, nbins, seed & (2**64 - 1), mode, integrand,
                                 p.ctypes.data if p.size else None, int(p.size), max_iters,
                                 d_workspace, ws_bytes, cuda_stream), "vegas_init_grid")
    return h.value


def vegas_set_config(h, block_threads=0, blocks_per_sm=0, min_samples_per_thread=0,
                     chunk_samples=0):
    cfg = vegas_config(block_threads, blocks_per_sm, min_samples_per_thread, chunk_samples)
    _check(lib().vegas_set_config(h, ctypes.byref(cfg)), "vegas_set_config")


def vegas_pipe_peak(op, iters, d_scratch, scratch_bytes, cuda_stream):
    """(lane-operations/s, SM MHz, SMs, blocks) of one VEGAS_PIPE_* operation."""
    out = np.zeros(4)
    _check(lib().vegas_pipe_peak(op, iters, d_scratch, scratch_bytes, cuda_stream,
                                 out.ctypes.data), "vegas_pipe_peak")
    return tuple(out)


def pipe_peaks(pipes=PIPES, reps=2, device="cuda", stream=None):
    """Measured peak of each named pipe on the current device: {name: {"per_s":
    lane-operations/s (best of `reps` launches), "sm_mhz": the SM clock during
    that launch, "per_sm_per_clk": per_s / (SMs x clock)}}."""
    import torch

    scratch = torch.zeros(VEGAS_PIPE_SCRATCH_BYTES, dtype=torch.uint8, device=device)
    st = stream if stream is not None else torch.cuda.current_stream(scratch.device)
    out = {}
    for name in pipes:
        best = max((vegas_pipe_peak(PIPES.index(name), 0, scratch.data_ptr(),
                                    VEGAS_PIPE_SCRATCH_BYTES, st.cuda_stream)
                    for _ in range(reps)), key=lambda r: r[0])
        rate, mhz, sms, _ = best
        out[name] = {"per_s": rate, "sm_mhz": mhz,
                     "per_sm_per_clk": rate / (sms * mhz * 1e6) if mhz > 0 else None}
    return out


def vegas_set_box(h, box):
    """box: [(lo_k, hi_k)] for each of the state's dimensions (the C call reads
    exactly dim of each; Vegas.set_box checks the shape)."""
    b = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(-1, 2))
    lo, hi = np.ascontiguousarray(b[:, 0]), np.ascontiguousarray(b[:, 1])
    _check(lib().vegas_set_box(h, lo.ctypes.data, hi.ctypes.data), "vegas_set_box")


def vegas_iterate(h, n_samples, adapt):
    _check(lib().vegas_iterate(h, int(n_samples), 1 if adapt else 0), "vegas_iterate")


def vegas_refine(h, alpha):
    _check(lib().vegas_refine(h, float(alpha)), "vegas_refine")


def vegas_result(h, first_iter=0):
    """(mean, sigma, chi2_dof, n_iter, nonfinite_seen)."""
    m, s, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_int()
    rc = lib().vegas_result(h, first_iter, ctypes.byref(m), ctypes.byref(s), ctypes.byref(c),
                            ctypes.byref(n))
    if rc not in (VEGAS_OK, VEGAS_ENONFINITE):
        raise VegasError(rc, "vegas_result")
    return m.value, s.value, c.value, n.value, rc == VEGAS_ENONFINITE


def vegas_result_range(h, first_iter, end_iter):
    """(mean, sigma, chi2_dof, nonfinite_seen) over iterations [first, end)."""
    m, s, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib().vegas_result_range(h, first_iter, end_iter, ctypes.byref(m), ctypes.byref(s),
                                  ctypes.byref(c))
    if rc not in (VEGAS_OK, VEGAS_ENONFINITE):
        raise VegasError(rc, "vegas_result_range")
    return m.value, s.value, c.value, rc == VEGAS_ENONFINITE


def vegas_get_iterations(h, max_rows=1 << 16):
    rows = np.zeros((max_rows, 6))
    n = ctypes.c_int()
    _check(lib().vegas_get_iterations(h, rows.ctypes.data, max_rows, ctypes.byref(n)),
           "vegas_get_iterations")
    return rows[: n.value].copy()


def vegas_get_iteration_times(h, max_rows=1 << 16):
    """Device time of each logged iteration in ns (numpy array)."""
    t = np.zeros(max_rows)
    n = ctypes.c_int()
    _check(lib().vegas_get_iteration_times(h, t.ctypes.data, max_rows, ctypes.byref(n)),
           "vegas_get_iteration_times")
    return t[: n.value].copy()


def vegas_get_grid(h, dim, nbins):
    e = np.empty((dim, nbins + 1))
    _check(lib().vegas_get_grid(h, e.ctypes.data), "vegas_get_grid")
    return e


def vegas_set_grid(h, edges):
    """edges: dim x (nbins + 1) doubles (the C call reads exactly that many;
    Vegas.set_grid checks the shape)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    _check(lib().vegas_set_grid(h, e.ctypes.data), "vegas_set_grid")


def vegas_get_histogram(h, dim, nbins):
    out = np.empty((dim, nbins))
    _check(lib().vegas_get_histogram(h, out.ctypes.data), "vegas_get_histogram")
    return out


def vegas_sample_words(seed, integral_id, it, i0, n, dim, d_out, cuda_stream):
    """Philox words of samples i0 .. i0+n-1 into the device buffer d_out (n x dim uint32)."""
    _check(lib().vegas_sample_words(seed & (2**64 - 1), integral_id, it, i0, n, dim, d_out,
                                    cuda_stream), "vegas_sample_words")


def vegas_iterate_noalloc(d_edges, dim, nbins, seed, it, mode, params, n_samples, adapt, alpha,
                          d_result, cuda_stream):
    """One Gaussian iteration without any device allocation (see include/vegas.h):
    d_edges (dim x (nbins+1) doubles) and d_result (6 doubles) are device
    addresses owned by the caller."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    _check(lib().vegas_iterate_noalloc(d_edges, dim, nbins, seed & (2**64 - 1), it, mode,
                                       p.ctypes.data, int(p.size), int(n_samples),
                                       1 if adapt else 0, float(alpha), d_result, cuda_stream),
           "vegas_iterate_noalloc")


def vegas_gauss_adjoint(h, params, it, n_samples, grad, d_out):
    """Fixed-grid Eq. 1 estimate (and its gradient in (mu, a) when grad) into
    the device buffer d_out of 2 (dim+2) + 1 doubles (see include/vegas.h)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    _check(lib().vegas_gauss_adjoint(h, p.ctypes.data, int(p.size), it, int(n_samples),
                                     1 if grad else 0, d_out), "vegas_gauss_adjoint")


def vegas_export_state(h):
    """The state's checkpoint blob (bytes)."""
    n = ctypes.c_size_t(0)
    _check(lib().vegas_export_state(h, None, ctypes.byref(n)), "vegas_export_state")
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().vegas_export_state(h, buf, ctypes.byref(n)), "vegas_export_state")
    return buf.raw[: n.value]


def vegas_import_state(blob, d_workspace, ws_bytes, cuda_stream):
    """A new state (handle) from a checkpoint blob."""
    h = ctypes.c_void_p(None)
    _check(lib().vegas_import_state(ctypes.byref(h), blob, len(blob), d_workspace, ws_bytes,
                                    cuda_stream), "vegas_import_state")
    return h.value


class vegas_user_integrand(ctypes.Structure):
    """The descriptor VEGAS_USER_INTEGRAND returns (include/vegas.h)."""
    _fields_ = [("dim", ctypes.c_int), ("args_bytes", ctypes.c_size_t),
                ("prepare", ctypes.c_void_p), ("launch", ctypes.c_void_p)]


def load_user_integrand(so_path, name):
    """Load a caller's integrand library (see build.build_user_integrand) and
    return (its CDLL, the address of descriptor `name`); keep the CDLL alive
    while a state uses the descriptor."""
    mod = ctypes.CDLL(so_path)
    fn = getattr(mod, name)
    fn.restype = ctypes.c_void_p
    fn.argtypes = []
    desc = fn()
    if not desc:
        raise VegasError(VEGAS_EINVAL, name)
    return mod, desc


def vegas_set_user_integrand(h, desc, d_data=0):
    _check(lib().vegas_set_user_integrand(h, desc, d_data or None), "vegas_set_user_integrand")


def vegas_destroy(h):
    if h:
        _check(lib().vegas_destroy(h), "vegas_destroy")


class Vegas:
    """One integration state on a CUDA device: torch owns the workspace and
    supplies the stream; the library does all the work."""

    def __init__(self, dim, nbins, seed, mode, integrand, params, max_iters=64, device="cuda",
                 stream=None):
        import torch

        self.dim, self.nbins, self.max_iters = dim, nbins, max_iters
        self.ws_bytes = vegas_workspace_bytes(dim, nbins, max_iters)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
        self.handle = vegas_init_grid(dim, nbins, seed, mode, integrand, params, max_iters,
                                      self.workspace.data_ptr(), self.ws_bytes,
                                      self.stream.cuda_stream)

    def config(self, **kw):
        vegas_set_config(self.handle, **kw)

    def set_box(self, box):
        """Integrate over [(lo_k, hi_k)] instead of the unit cube (before the
        first iteration)."""
        b = np.asarray(box, dtype=np.float64)
        if b.shape != (self.dim, 2):
            raise ValueError(f"box must be {self.dim} (lo, hi) pairs, got shape {b.shape}")
        vegas_set_box(self.handle, b)

    def inject_failure(self, countdown):
        """Testing hook: the countdown-th next iterate/refine call fails with
        VEGAS_ECUDA before enqueueing anything (0 cancels)."""
        _check(lib().vegas_inject_failure(self.handle, int(countdown)), "vegas_inject_failure")

    def set_user_integrand(self, desc, data=None, module=None):
        """Attach a VEGAS_USER_INTEGRAND descriptor (an address, e.g. from
        load_user_integrand) to a VEGAS_USER state; `data` is an optional
        device tensor whose pointer the integrand receives (kept alive with
        `module`, the integrand's library, as long as this state)."""
        vegas_set_user_integrand(self.handle, desc, data.data_ptr() if data is not None else 0)
        self._user_refs = (data, module)

    def export_state(self):
        return vegas_export_state(self.handle)

    @classmethod
    def from_state(cls, blob, device="cuda", stream=None):
        """Resume a state from vegas_export_state's blob (header words: dim at
        offset 16, nbins at 24, max_iters at 48)."""
        import struct

        import torch

        dim, nbins = struct.unpack_from("<QQ", blob, 16)
        (max_iters,) = struct.unpack_from("<Q", blob, 48)
        self = cls.__new__(cls)
        self.dim, self.nbins, self.max_iters = int(dim), int(nbins), int(max_iters)
        self.ws_bytes = vegas_workspace_bytes(self.dim, self.nbins, int(max_iters))
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(
            self.workspace.device)
        self.handle = vegas_import_state(blob, self.workspace.data_ptr(), self.ws_bytes,
                                         self.stream.cuda_stream)
        return self

    def iterate(self, n, adapt):
        vegas_iterate(self.handle, n, adapt)

    def refine(self, alpha=1.5):
        vegas_refine(self.handle, alpha)

    def result(self, first_iter=0):
        return vegas_result(self.handle, first_iter)

    def iterations(self):
        return vegas_get_iterations(self.handle, self.max_iters)

    def records(self, first_iter=0):
        """One record per logged iteration t >= first_iter: its samples, I,
        sigma (= sqrt(var)), non-finite count, device time (ms) and rate, and
        the combined result over iterations first_iter .. t (the running
        estimate, its sigma and chi^2 per degree of freedom)."""
        rows, ns = self.iterations(), self.iteration_times()
        out = []
        for t in range(first_iter, len(rows)):
            mean, sigma, chi2, _ = vegas_result_range(self.handle, first_iter, t + 1)
            ms = ns[t] / 1e6
            out.append({"iter": t, "n": int(rows[t][2]), "I": rows[t][4],
                        "sigma": math.sqrt(rows[t][5]), "nonfinite": int(rows[t][3]),
                        "device_ms": ms, "samples_per_s": rows[t][2] / (ms / 1e3) if ms > 0 else None,
                        "mean_so_far": mean, "sigma_so_far": sigma, "chi2_dof_so_far": chi2})
        return out

    def iteration_times(self):
        """Device time of each logged iteration, ns."""
        return vegas_get_iteration_times(self.handle, self.max_iters)

    def grid(self):
        return vegas_get_grid(self.handle, self.dim, self.nbins)

    def set_grid(self, edges):
        e = np.asarray(edges, dtype=np.float64)
        if e.shape != (self.dim, self.nbins + 1):
            raise ValueError(f"edges must have shape {(self.dim, self.nbins + 1)}, got {e.shape}")
        vegas_set_grid(self.handle, e)

    def histogram(self):
        return vegas_get_histogram(self.handle, self.dim, self.nbins)

    def gauss_adjoint(self, params, it, n, grad=True):
        """(I, dI/dmu, dI/da, variances, nonfinite) on the current grid as a
        device tensor of 2 (dim+2) + 1 doubles."""
        import torch

        out = torch.empty(2 * (self.dim + 2) + 1, dtype=torch.float64,
                          device=self.workspace.device)
        vegas_gauss_adjoint(self.handle, params, it, n, grad, out.data_ptr())
        return out

    def run(self, schedule, alpha=1.5):
        """Enqueue (n, adapt) iterations; each adapting one is followed by a
        refinement.  Asynchronous."""
        for n, adapt in schedule:
            self.iterate(n, adapt)
            if adapt:
                self.refine(alpha)

    def capture(self, schedule, alpha=1.5):
        """A CUDA graph of run(schedule), captured on this state's stream,
        which must not be the default stream (nothing runs during the
        capture).  Each replay() launches it on that stream and runs the
        schedule as further iterations with fresh counters, from the grid it
        finds; the log's capacity (max_iters) bounds the replays."""
        import torch

        if self.stream.cuda_stream == 0:
            raise ValueError("capture needs a state created on a non-default stream")
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=self.stream):
            self.run(schedule, alpha)
        return StateGraph(graph, self.stream)

    def close(self):
        if self.handle:
            vegas_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def integrate(integrand, params, dim, n_iter, n_events, adapt_iters=None, nbins=50,
              mode=VEGAS_FP32_EVAL, seed=1, alpha=1.5, box=None, stream=None):
    """One call from integrand to result, the shape of the paper's wrapper
    (integrand, dimension, iterations, events per iteration): n_iter
    iterations of n_events samples, of which the first adapt_iters (default:
    all but the last, at least one) adapt the grid; returns (mean, sigma,
    chi2_dof) combined over the iterations on the frozen grid, or over all of
    them when every iteration adapts."""
    if n_iter < 1:
        raise ValueError("n_iter must be >= 1")
    k = max(1, n_iter - 1) if adapt_iters is None else int(adapt_iters)
    v = Vegas(dim, nbins, seed, mode, integrand, params, max_iters=n_iter, stream=stream)
    try:
        if box is not None:
            v.set_box(box)
        v.run([(n_events, 1)] * k + [(n_events, 0)] * (n_iter - k), alpha)
        mean, sigma, chi2, _, _ = v.result(k if k < n_iter else 0)
    finally:
        v.close()
    return mean, sigma, chi2


class StateGraph:
    """A captured schedule of one state (Vegas.capture); replay() launches it
    on the state's stream."""

    def __init__(self, graph, stream):
        self.graph, self.stream = graph, stream

    def replay(self):
        import torch

        with torch.cuda.stream(self.stream):
            self.graph.replay()


# ---------------------------------------------------------------- batches
def _batch_arrays(dims, n_samples, params_list):
    dims_a = np.ascontiguousarray(dims, dtype=np.int32)
    n_a = np.ascontiguousarray(n_samples, dtype=np.uint64)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64)
                                                for p in params_list]))
    return dims_a, n_a, flat


def vegas_batch_workspace_bytes(dims, n_samples, nbins, max_iters):
    dims_a, n_a, _ = _batch_arrays(dims, n_samples, [[0.0]])
    out = ctypes.c_size_t(0)
    _check(lib().vegas_batch_workspace_bytes(len(dims_a), dims_a.ctypes.data, n_a.ctypes.data,
                                             nbins, max_iters, ctypes.byref(out)),
           "vegas_batch_workspace_bytes")
    return out.value


def vegas_batch_init(dims, n_samples, nbins, seed, mode, params_list, max_iters, d_workspace,
                     ws_bytes, cuda_stream, integrand=VEGAS_GAUSS, boxes=None):
    """A batch handle.  integrand: one built-in id for every integral;
    params_list: each integral's parameters in that integrand's layout;
    boxes: None, or each integral's [(lo_k, hi_k)] (None entries: unit cube)."""
    params_list = [p if p is not None else [] for p in params_list]
    if len(params_list) != len(dims) or (boxes is not None and len(boxes) != len(dims)):
        raise ValueError("need one parameter list (and one box, if any) per integral")
    for d, p in zip(dims, params_list):  # the C call reads exactly these counts
        need = {VEGAS_GAUSS: 1 + d, VEGAS_GAUSS_MIX2: 1 + 2 * d, VEGAS_GENZ_DISC: 2 * d,
                VEGAS_GENZ_PPEAK: 2 * d}.get(integrand, 0)
        if len(p) != need:
            raise ValueError(f"integrand {integrand} in dimension {d} takes {need} "
                             f"parameters, got {len(p)}")
    dims_a, n_a, flat = _batch_arrays(dims, n_samples, params_list)
    lo = hi = None
    if boxes is not None:
        rows = [np.asarray(bx if bx is not None else [(0.0, 1.0)] * d, dtype=np.float64)
                .reshape(d, 2) for bx, d in zip(boxes, dims_a)]
        both = np.concatenate(rows)
        lo, hi = np.ascontiguousarray(both[:, 0]), np.ascontiguousarray(both[:, 1])
    h = ctypes.c_void_p(None)
    _check(lib().vegas_batch_init_integrand(
        ctypes.byref(h), len(dims_a), dims_a.ctypes.data, n_a.ctypes.data, nbins,
        seed & (2**64 - 1), mode, integrand, flat.ctypes.data if flat.size else None,
        lo.ctypes.data if lo is not None else None, hi.ctypes.data if hi is not None else None,
        max_iters, d_workspace, ws_bytes, cuda_stream), "vegas_batch_init_integrand")
    return h.value


class VegasBatch:
    """Many integrals of one built-in integrand family (default: the Eq. 1
    Gaussian) advanced together, one persistent launch per iteration, each over
    the unit cube or its own box; torch owns the workspace and supplies the
    stream."""

    def __init__(self, dims, n_samples, nbins, seed, mode, params_list, max_iters=16,
                 device="cuda", stream=None, integrand=VEGAS_GAUSS, boxes=None):
        import torch

        self.dims = [int(d) for d in dims]
        self.n_samples = [int(n) for n in n_samples]
        self.nbins, self.max_iters = nbins, max_iters
        self.mode, self.integrand = mode, integrand
        self.ws_bytes = vegas_batch_workspace_bytes(self.dims, n_samples, nbins, max_iters)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(
            self.workspace.device)
        self.handle = vegas_batch_init(self.dims, n_samples, nbins, seed, mode, params_list,
                                       max_iters, self.workspace.data_ptr(), self.ws_bytes,
                                       self.stream.cuda_stream, integrand, boxes)

    def config(self, block_threads=0, tile_samples=0):
        _check(lib().vegas_batch_set_config(self.handle, block_threads, tile_samples),
               "vegas_batch_set_config")

    def config_tiles_by_dim(self, tiles):
        """Samples per tile by dimension: {dim: samples} (0 or absent: the
        set_config size); an empty dict clears them."""
        arr = (ctypes.c_uint64 * VEGAS_MAX_DIM)()
        for d, t in tiles.items():
            arr[int(d) - 1] = int(t)
        _check(lib().vegas_batch_set_tiles_by_dim(self.handle, arr, VEGAS_MAX_DIM),
               "vegas_batch_set_tiles_by_dim")

    def set_stream(self, stream):
        self.stream = stream
        _check(lib().vegas_batch_set_stream(self.handle, stream.cuda_stream),
               "vegas_batch_set_stream")

    def reset(self):
        _check(lib().vegas_batch_reset(self.handle), "vegas_batch_reset")

    def iterate(self, adapt=True, alpha=1.5):
        _check(lib().vegas_batch_iterate(self.handle, 1 if adapt else 0, float(alpha)),
               "vegas_batch_iterate")

    def run(self, iters, adapt=True, alpha=1.5):
        """Reset, then `iters` iterations (asynchronous)."""
        self.reset()
        for _ in range(iters):
            self.iterate(adapt, alpha)

    def capture(self, iters, adapt=True, alpha=1.5):
        """A CUDA graph of reset + `iters` iterations, captured on a side stream;
        replay() runs the whole schedule again."""
        import torch

        side = torch.cuda.Stream(device=self.workspace.device)
        side.wait_stream(torch.cuda.current_stream(self.workspace.device))
        old = self.stream
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            self.set_stream(side)
            self.run(iters, adapt, alpha)  # warm-up outside the capture
            side.synchronize()
            with torch.cuda.graph(graph, stream=side):
                self.run(iters, adapt, alpha)
        torch.cuda.current_stream(self.workspace.device).wait_stream(side)
        self.set_stream(old)
        return graph

    def result(self, index, first_iter=0):
        m, s, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int()
        rc = lib().vegas_batch_result(self.handle, index, first_iter, ctypes.byref(m),
                                      ctypes.byref(s), ctypes.byref(c), ctypes.byref(n))
        if rc not in (VEGAS_OK, VEGAS_ENONFINITE):
            raise VegasError(rc, "vegas_batch_result")
        return m.value, s.value, c.value, n.value, rc == VEGAS_ENONFINITE

    def log(self):
        out = np.zeros((len(self.dims), self.max_iters, 6))
        _check(lib().vegas_batch_get_log(self.handle, out.ctypes.data), "vegas_batch_get_log")
        return out

    def grid(self, index):
        e = np.empty((self.dims[index], self.nbins + 1))
        _check(lib().vegas_batch_get_grid(self.handle, index, e.ctypes.data),
               "vegas_batch_get_grid")
        return e

    def histogram(self, index):
        """The (f J)^2 histogram integral `index`'s last refinement used."""
        h = np.empty((self.dims[index], self.nbins))
        _check(lib().vegas_batch_get_histogram(self.handle, index, h.ctypes.data),
               "vegas_batch_get_histogram")
        return h

    def close(self):
        if self.handle:
            _check(lib().vegas_batch_destroy(self.handle), "vegas_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(dim, nbins, mode, integrand, params, n, adapt=False, blocks=(128, 256),
             blocks_per_sm=(0, 2, 3), min_samples=(8, 64), reps=3, device="cuda"):
    """Pick a launch configuration (vegas_set_config) for iterations of n
    samples of this shape by timing `reps` iterations per candidate on a
    scratch state (CUDA events, best of reps).  Samples depend only on their
    counters, so the choice changes speed, never results.  Returns
    (best config as a dict for Vegas.config, {candidate: ms})."""
    import itertools

    import torch

    timings = {}
    for bt, bps, ms in itertools.product(blocks, blocks_per_sm, min_samples):
        v = Vegas(dim, nbins, 1, mode, integrand, params, max_iters=reps + 1, device=device)
        try:
            v.config(block_threads=bt, blocks_per_sm=bps, min_samples_per_thread=ms)
            v.iterate(n, adapt)  # warm-up
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(v.stream)
                v.iterate(n, adapt)
                e1.record(v.stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            timings[(bt, bps, ms)] = best
        finally:
            v.close()
    bt, bps, ms = min(timings, key=timings.get)
    return dict(block_threads=bt, blocks_per_sm=bps, min_samples_per_thread=ms), timings


class TuningTable:
    """Tuned launch configurations kept in a JSON file, keyed by (mode,
    integrand, dim, nbins, adapt, n bucket) -- the bucket is the power of ten
    of the iteration's sample count -- so that a shape tuned once is not tuned
    again in a later process.  lookup() returns the stored configuration or
    runs `tuner` (autotune by default), stores and saves its choice."""

    def __init__(self, path, tuner=None):
        import json

        self.path, self.tuner = path, tuner or autotune
        self.entries = {}
        if os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    @staticmethod
    def key(mode, integrand, dim, nbins, n, adapt):
        bucket = len(str(int(n))) - 1  # floor(log10 n)
        return f"mode={mode},integrand={integrand},d={dim},N={nbins},adapt={int(bool(adapt))}," \
               f"n=1e{bucket}"

    def lookup(self, dim, nbins, mode, integrand, params, n, adapt=False, **tuner_kw):
        k = self.key(mode, integrand, dim, nbins, n, adapt)
        if k not in self.entries:
            cfg, _ = self.tuner(dim, nbins, mode, integrand, params, n, adapt=adapt, **tuner_kw)
            self.entries[k] = {name: int(v) for name, v in cfg.items()}
            self._save()
        return dict(self.entries[k])

    def _save(self):
        import json

        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    @staticmethod
    def batch_key(batch):
        """A batch's key: mode, integrand, bins, integral count, the dimension
        buckets it spans and the decade of its samples per iteration."""
        spans = sorted({f"{lo}-{hi}" for lo, hi in DIM_BUCKETS for d in batch.dims
                        if lo <= d <= hi})
        total = len(str(int(sum(batch.n_samples)))) - 1
        return (f"batch,mode={batch.mode},integrand={batch.integrand},N={batch.nbins},"
                f"count={len(batch.dims)},buckets={'+'.join(spans)},n=1e{total}")

    def lookup_batch(self, batch, tuner=None, **tuner_kw):
        """Configure `batch` from its stored entry -- block size, batch-wide
        tile and one tile per dimension bucket -- tuning it first (with
        `tuner`, autotune_batch by default) if its key is new.  Returns the
        entry."""
        k = self.batch_key(batch)
        if k not in self.entries:
            (bt, ts, by_dim), _ = (tuner or autotune_batch)(batch, **tuner_kw)
            by_bucket = {}
            for lo, hi in DIM_BUCKETS:
                got = {by_dim[d] for d in range(lo, hi + 1) if d in by_dim}
                if got:
                    by_bucket[f"{lo}-{hi}"] = int(got.pop())
            self.entries[k] = {"block_threads": int(bt), "tile_samples": int(ts),
                               "tiles_by_bucket": by_bucket}
            self._save()
        e = self.entries[k]
        batch.config(block_threads=e["block_threads"], tile_samples=e["tile_samples"])
        tiles = {}
        for span, t in e["tiles_by_bucket"].items():
            lo, hi = (int(x) for x in span.split("-"))
            tiles.update({d: t for d in set(batch.dims) if lo <= d <= hi})
        batch.config_tiles_by_dim(tiles)
        batch.reset()
        return dict(e)


DIM_BUCKETS = ((1, 4), (5, 8), (9, 12), (13, 16), (17, 20))


def autotune_batch(batch, blocks=(128, 256, 512),
                   samples_per_thread=(1, 2, 4, 8, 16, 32, 64, 128, 256, 512), tiles=None,
                   reps=2, alpha=1.5, buckets=DIM_BUCKETS):
    """Pick the launch configuration of a batch by timing one adapting
    iteration of every integral per candidate (CUDA events on the batch's
    stream, best of `reps`).  First the batch-wide (block_threads,
    tile_samples): every block size in `blocks` with every samples-per-thread
    count s in `samples_per_thread` (tile = block x s, at least 128 samples),
    or with every size in `tiles` when that is given.  Then, one dimension
    bucket at a time, a tile size for the integrals of that bucket (half or
    twice the batch's, kept if faster).  The samples are functions of their
    counters, so the choice changes speed, never results.  Leaves the batch
    configured with the winner and reset; returns ((block_threads,
    tile_samples, {dim: tile}), {candidate: ms})."""
    import torch

    def time_one():
        best = float("inf")
        for _ in range(reps):
            batch.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(batch.stream)
            batch.iterate(True, alpha)
            e1.record(batch.stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    timings = {}
    batch.config_tiles_by_dim({})
    for bt in blocks:
        sizes = tiles if tiles is not None else sorted({max(128, bt * s) for s in
                                                        samples_per_thread})
        for ts in sizes:
            batch.config(block_threads=bt, tile_samples=ts)
            timings[(bt, ts)] = time_one()
    bt, ts = min(timings, key=timings.get)
    batch.config(block_threads=bt, tile_samples=ts)
    best_ms, by_dim = timings[(bt, ts)], {}
    present = set(batch.dims)
    for lo, hi in buckets:
        dims = [d for d in range(lo, hi + 1) if d in present]
        if not dims:
            continue
        for cand in (ts // 2, ts * 2):
            if cand < 128:
                continue
            trial = {**by_dim, **{d: cand for d in dims}}
            batch.config_tiles_by_dim(trial)
            ms = time_one()
            timings[(bt, ts, (lo, hi), cand)] = ms
            if ms < best_ms:
                best_ms, by_dim = ms, trial
        batch.config_tiles_by_dim(by_dim)
    batch.reset()
    return (bt, ts, by_dim), timings
