"""Python binding of libfsc.so, the GB300 fast spectral clustering library.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (PyTorch provides device memory and
streams); the calls mirror the C ABI in ``include/fsc.h``:

    g = Graph(row_ptr, col, w)                  # fsc_create_graph
    emb = embed(g, l, t, seed)                  # fsc_embed
    labels, st = kmeans(emb, l, k, seed)        # fsc_kmeans
    labels, st = cluster(g, k, l, t, seed)      # fsc_cluster

There is no CPU fallback: importing works without a GPU (so the library's
exports can be inspected), but every call needs the built ``libfsc.so`` and a
CUDA device, and raises otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

__all__ = [
    "FscError", "Graph", "KmeansStats", "EmbedOpts", "lib", "embed", "power_step", "kmeans", "cluster",
    "default_params", "pad_l", "sync_status", "set_wait_limit_ns", "inject_barrier_stall", "status_string", "LIB_PATH",
    "F32", "BF16", "F16", "FILTER_NO_FALLBACK", "release_cached_memory", "VALIDATE_SYMMETRY", "COPY", "EMBED_RESCALE", "BATCH_AUTOTUNE", "Batch", "autotune",
    "knn_graph", "embed_orthogonal", "top_eigenvectors", "kmeans_best", "partition_scores", "filter_embed", "cluster_filtered", "mlp_forward", "mlp_train_step", "load_filter_params", "NPARAM",
]

# FSC_LIBRARY=checked selects the build with index checks (build.py --bounds-check)
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "libfsc_checked.so" if os.environ.get("FSC_LIBRARY") == "checked" else "libfsc.so")

F32, BF16, F16 = 0, 1, 2
FILTER_NO_FALLBACK = 0x100
VALIDATE_SYMMETRY = 0x1
COPY = 0x4
EMBED_RESCALE = 0x1
BATCH_AUTOTUNE = 0x2

_STATUS = {
    0: "FSC_OK", 1: "FSC_ERR_INVALID_ARG", 2: "FSC_ERR_INDEX_RANGE", 3: "FSC_ERR_NOT_SYMMETRIC",
    4: "FSC_ERR_SELF_LOOP", 5: "FSC_ERR_BAD_WEIGHT", 6: "FSC_ERR_OOM", 7: "FSC_ERR_CUDA",
    8: "FSC_ERR_TIMEOUT", 9: "FSC_ERR_UNSORTED", 10: "FSC_ERR_TOO_LARGE",
}


class FscError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        self.name = _STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name} ({status_string(status)})")


class EmbedOpts(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("threads_per_row", C.c_int32),
                ("ev_spmm_begin", C.c_void_p), ("ev_spmm_end", C.c_void_p)]


class KmeansStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("changed", C.c_int32), ("empty_events", C.c_int32),
                ("device_status", C.c_int32), ("inertia", C.c_double), ("seeding_potential", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class FilterReport(C.Structure):
    _fields_ = [("energy_ratio", C.c_double), ("threshold", C.c_double), ("fallback", C.c_int32),
                ("fallback_t", C.c_int32)]


class BatchDesc(C.Structure):
    _fields_ = [("num_graphs", C.c_int32), ("vertex_offset", C.c_void_p), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("w", C.c_void_p), ("k", C.c_void_p), ("l", C.c_void_p),
                ("t", C.c_void_p), ("seed", C.c_void_p), ("labels", C.c_void_p), ("store", C.c_int32),
                ("max_iter", C.c_int32), ("flags", C.c_uint32)]


class GraphInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("n_isolated", C.c_int64), ("weighted", C.c_int32),
                ("volume", C.c_double), ("deg", C.c_void_p), ("dinv", C.c_void_p), ("invdeg", C.c_void_p),
                ("deg_sumsq", C.c_double), ("deg_max", C.c_double)]


_lib = None


def lib() -> C.CDLL:
    """The loaded libfsc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfsc.so not built at {LIB_PATH}; run `python -m paper_2310_10939_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, u32, u64 = C.c_void_p, C.c_int64, C.c_int, C.c_uint32, C.c_uint64
        L.fsc_create_graph.argtypes = [i64, i64, vp, vp, vp, u32, vp, C.POINTER(vp)]
        L.fsc_destroy_graph.argtypes = [vp]
        L.fsc_graph_info.argtypes = [vp, C.POINTER(GraphInfo)]
        L.fsc_pad_l.argtypes = [i32]
        L.fsc_pad_l.restype = i32
        L.fsc_embed.argtypes = [vp, i32, i32, u64, i32, vp, C.POINTER(EmbedOpts), vp]
        L.fsc_power_step.argtypes = [vp, i32, i32, vp, vp, i32, vp]
        L.fsc_gather_floor.argtypes = [vp, i32, i32, vp, vp, vp]
        L.fsc_gather_floor.restype = i32
        L.fsc_bounds_report.argtypes = [C.POINTER(i32), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), i32]
        L.fsc_bounds_report.restype = i32
        L.fsc_kmeans.argtypes = [vp, i64, i32, i32, i32, u64, i32, vp, vp, vp, C.POINTER(KmeansStats), vp]
        L.fsc_kmeans_static.argtypes = [vp, i64, i32, i32, i32, u64, i32, vp, vp, vp, C.POINTER(KmeansStats), vp]
        L.fsc_knn_graph.argtypes = [vp, i64, i32, i32, vp, vp, vp, i64, C.POINTER(i64), C.POINTER(C.c_double), vp]
        L.fsc_knn_graph.restype = i32
        L.fsc_embed_orthogonal.argtypes = [vp, i32, i32, i32, u64, vp, C.POINTER(EmbedOpts), vp]
        L.fsc_embed_orthogonal.restype = i32
        L.fsc_top_eigenvectors.argtypes = [vp, i32, i32, i32, u64, vp, C.POINTER(C.c_double), C.POINTER(EmbedOpts), vp]
        L.fsc_top_eigenvectors.restype = i32
        L.fsc_kmeans_best.argtypes = [vp, i64, i32, i32, i32, u64, i32, i32, vp, vp, vp, C.POINTER(KmeansStats),
                                      C.POINTER(i32), vp]
        L.fsc_kmeans_best.restype = i32
        L.fsc_partition_scores.argtypes = [vp, vp, i64, i32, i32, C.POINTER(C.c_double), vp]
        L.fsc_partition_scores.restype = i32
        L.fsc_kmeans_static.restype = i32
        L.fsc_cluster.argtypes = [vp, i32, i32, i32, u64, i32, i32, vp, C.POINTER(KmeansStats),
                                  C.POINTER(EmbedOpts), vp]
        L.fsc_autotune.argtypes = [vp, i32, i32, C.POINTER(i32), C.POINTER(C.c_float), vp]
        L.fsc_batch_create.argtypes = [C.POINTER(BatchDesc), vp, C.POINTER(vp)]
        L.fsc_batch_run.argtypes = [vp, vp]
        L.fsc_batch_results.argtypes = [vp, vp, vp, vp, vp]
        L.fsc_batch_destroy.argtypes = [vp]
        L.fsc_batch_embedding.argtypes = [vp, i32, vp, vp]
        for name in ("fsc_autotune", "fsc_batch_create", "fsc_batch_run", "fsc_batch_results", "fsc_batch_destroy",
                     "fsc_batch_embedding"):
            getattr(L, name).restype = i32
        L.fsc_filter_embed.argtypes = [vp, i32, i32, u64, i32, vp, vp, vp, vp, vp, vp, C.POINTER(EmbedOpts), vp]
        L.fsc_cluster_filtered.argtypes = [vp, i32, i32, u64, i32, vp, i32, vp, C.POINTER(KmeansStats),
                                           C.POINTER(FilterReport), C.POINTER(EmbedOpts), vp]
        L.fsc_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
        L.fsc_mlp_train_step.argtypes = [vp, vp, vp, vp, i32, C.c_float, C.c_float, vp, vp, vp, i32, vp, i32, vp]
        for name in ("fsc_filter_embed", "fsc_cluster_filtered", "fsc_mlp_forward", "fsc_mlp_train_step"):
            getattr(L, name).restype = i32
        L.fsc_default_params.argtypes = [i64, i32, i32, C.POINTER(i32), C.POINTER(i32)]
        L.fsc_sync_status.argtypes = [vp]
        L.fsc_release_cached_memory.argtypes = []
        L.fsc_release_cached_memory.restype = i32
        L.fsc_set_wait_limit_ns.argtypes = [i64]
        L.fsc_set_wait_limit_ns.restype = None
        L.fsc_inject_barrier_stall.argtypes = [i32]
        L.fsc_inject_barrier_stall.restype = None
        L.fsc_status_string.argtypes = [i32]
        L.fsc_status_string.restype = C.c_char_p
        L.fsc_version.restype = C.c_char_p
        for name in ("fsc_create_graph", "fsc_destroy_graph", "fsc_graph_info", "fsc_embed", "fsc_power_step",
                     "fsc_kmeans", "fsc_cluster", "fsc_default_params", "fsc_sync_status"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().fsc_status_string(int(status)).decode()
    except ImportError:
        return _STATUS.get(status, "?")


def _check(rc: int, where: str):
    if rc != 0:
        raise FscError(rc, where)


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _require_cuda(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor of dtype {dtype}")


def pad_l(l: int) -> int:
    return int(lib().fsc_pad_l(int(l)))


def default_params(n: int, k: int, mode: int = 0):
    l, t = C.c_int(), C.c_int()
    _check(lib().fsc_default_params(int(n), int(k), int(mode), C.byref(l), C.byref(t)), "fsc_default_params")
    return l.value, t.value


def sync_status(stream=None):
    _check(lib().fsc_sync_status(_stream(stream)), "fsc_sync_status")


def release_cached_memory():
    """fsc_release_cached_memory: return the library pool's cached device blocks to the driver."""
    _check(lib().fsc_release_cached_memory(), "fsc_release_cached_memory")


def set_wait_limit_ns(ns: int):
    lib().fsc_set_wait_limit_ns(int(ns))


def inject_barrier_stall(enable: bool):
    """Testing hook: grid barriers are never released, so every wait runs into its limit."""
    lib().fsc_inject_barrier_stall(1 if enable else 0)


class Graph:
    """A CSR graph on the GPU with its degrees (fsc_create_graph).  Keeps the CSR tensors alive, or
    with ``copy=True`` lets the library keep its own copy (FSC_COPY) and holds no reference to them."""

    def __init__(self, row_ptr, col, w=None, validate_symmetry: bool = False, stream=None, copy: bool = False):
        torch = _torch()
        _require_cuda(row_ptr, torch.int64, "row_ptr")
        _require_cuda(col, torch.int32, "col")
        if w is not None:
            _require_cuda(w, torch.float32, "w")
        self.device = row_ptr.device
        self.n = row_ptr.numel() - 1
        self.nnz = col.numel()
        h = C.c_void_p()
        flags = (VALIDATE_SYMMETRY if validate_symmetry else 0) | (COPY if copy else 0)
        _check(lib().fsc_create_graph(self.n, self.nnz, _ptr(row_ptr), _ptr(col), _ptr(w), flags,
                                      _stream(stream), C.byref(h)), "fsc_create_graph")
        self.handle = h
        self.row_ptr, self.col, self.w = (None, None, None) if copy else (row_ptr, col, w)

    @classmethod
    def from_workload(cls, g, device="cuda", **kw):
        """Upload a ``workloads.Graph`` (numpy CSR) and wrap it."""
        torch = _torch()
        rp = torch.as_tensor(g.row_ptr, device=device)
        col = torch.as_tensor(g.col, device=device)
        w = None if g.w is None else torch.as_tensor(g.w, device=device)
        return cls(rp, col, w, **kw)

    def info(self) -> dict:
        inf = GraphInfo()
        _check(lib().fsc_graph_info(self.handle, C.byref(inf)), "fsc_graph_info")
        return {f: getattr(inf, f) for f, _ in GraphInfo._fields_}

    def degrees(self):
        """Copy of the library's float64 degree array d(v) (device tensor)."""
        return _wrap_device(self.info()["deg"], (self.n,), "<f8").clone()

    def dinv(self):
        """Copy of the library's float32 D^-1/2 diagonal (device tensor)."""
        return _wrap_device(self.info()["dinv"], (self.n,), "<f4").clone()

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().fsc_destroy_graph(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _wrap_device(ptr: int, shape, typestr: str):
    """Zero-copy torch view of library-owned device memory (valid while the owner lives)."""
    return _torch().as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")


def _opts(rescale=False, threads_per_row=0, events=None):
    o = EmbedOpts()
    o.flags = EMBED_RESCALE if rescale else 0
    o.threads_per_row = int(threads_per_row)
    if events is not None:
        for ev in events:
            if not ev.cuda_event:          # torch creates the CUDA event lazily on first record
                ev.record()
        o.ev_spmm_begin = events[0].cuda_event
        o.ev_spmm_end = events[1].cuda_event
    return o


def embed(g: Graph, l: int, t: int, seed: int, store: int = F32, out=None, rescale: bool = False,
          threads_per_row: int = 0, events=None, stream=None):
    """fsc_embed: returns (or fills) an n x pad_l(l) float32 CUDA tensor = D^-1/2 M^t X0."""
    torch = _torch()
    lp = pad_l(l)
    if out is None:
        out = torch.empty((g.n, max(lp, 1)), dtype=torch.float32, device=g.device)
    _require_cuda(out, torch.float32, "out")
    o = _opts(rescale, threads_per_row, events)
    _check(lib().fsc_embed(g.handle, int(l), int(t), int(seed) & (2**64 - 1), int(store), _ptr(out),
                           C.byref(o), _stream(stream)), "fsc_embed")
    return out


def power_step(g: Graph, l: int, z_in, z_out, store: int = F32, threads_per_row: int = 0, stream=None):
    """fsc_power_step: z_out = (z_in + D^-1 A z_in) / 2 (one iteration in embedding coordinates)."""
    _check(lib().fsc_power_step(g.handle, int(l), int(store), _ptr(z_in), _ptr(z_out), int(threads_per_row),
                                _stream(stream)), "fsc_power_step")
    return z_out


def bounds_report(clear: bool = False):
    """fsc_bounds_report: None if nothing was recorded, -1 if the library has no index checks, else
    (site, index, lo, hi) of the first out-of-range index."""
    site, idx, lo, hi = C.c_int(0), C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _check(lib().fsc_bounds_report(C.byref(site), C.byref(idx), C.byref(lo), C.byref(hi), 1 if clear else 0),
           "fsc_bounds_report")
    if site.value == 0:
        return None
    if site.value < 0:
        return -1
    return site.value, idx.value, lo.value, hi.value


def gather_floor(g: Graph, l: int, z, store: int = F32, out=None, stream=None):
    """fsc_gather_floor: the neighbour gathers of one power step with no row structure (a
    measurement aid; the returned device float means nothing)."""
    torch = _torch()
    if out is None:
        out = torch.empty(1, dtype=torch.float32, device=z.device)
    _check(lib().fsc_gather_floor(g.handle, l, store, _ptr(z), _ptr(out), _stream(stream)), "fsc_gather_floor")
    return out


def kmeans(emb, l: int, k: int, seed: int, max_iter: int = 100, labels=None, want_centroids: bool = False,
           want_seeds: bool = False, sync: bool = True, stream=None):
    """fsc_kmeans on the rows of ``emb`` (n x ld float32).  Returns (labels, stats, centroids, seeds)."""
    torch = _torch()
    _require_cuda(emb, torch.float32, "emb")
    n, ld = emb.shape
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=emb.device)
    cen = torch.empty((k, l), dtype=torch.float64, device=emb.device) if want_centroids else None
    sd = torch.empty(k, dtype=torch.int64, device=emb.device) if want_seeds else None
    st = KmeansStats()
    _check(lib().fsc_kmeans(_ptr(emb), n, int(l), int(ld), int(k), int(seed) & (2**64 - 1), int(max_iter),
                            _ptr(labels), _ptr(cen), _ptr(sd), C.byref(st) if sync else None, _stream(stream)),
           "fsc_kmeans")
    return labels, (st.as_dict() if sync else None), cen, sd


def knn_graph(points, knn: int, weighted: bool = True, stream=None):
    """fsc_knn_graph: the union-symmetrised kNN graph of float32 CUDA points (n x dim).
    Returns (row_ptr int64, col int32, w float32 or None, sigma) CUDA tensors (col, w trimmed)."""
    torch = _torch()
    _require_cuda(points, torch.float32, "points")
    n, dim = points.shape
    cap = 2 * n * int(knn)
    rp = torch.empty(n + 1, dtype=torch.int64, device=points.device)
    col = torch.empty(cap, dtype=torch.int32, device=points.device)
    w = torch.empty(cap, dtype=torch.float32, device=points.device) if weighted else None
    nnz = C.c_int64(0)
    sig = C.c_double(0.0)
    _check(lib().fsc_knn_graph(_ptr(points), int(n), int(dim), int(knn), _ptr(rp), _ptr(col), _ptr(w), int(cap),
                               C.byref(nnz), C.byref(sig), _stream(stream)), "fsc_knn_graph")
    m = int(nnz.value)
    return rp, col[:m], (w[:m] if w is not None else None), float(sig.value)


def embed_orthogonal(g: Graph, l: int, t: int, seed: int, every: int = 1, out=None, threads_per_row: int = 0,
                     events=None, stream=None):
    """fsc_embed_orthogonal: orthogonal iteration (the power method on a block kept D-orthonormal);
    returns (or fills) the n x pad_l(l) float32 embedding D^-1/2 Q."""
    torch = _torch()
    if out is None:
        out = torch.empty((g.n, pad_l(l)), dtype=torch.float32, device=g.device)
    _require_cuda(out, torch.float32, "out")
    o = _opts(False, threads_per_row, events)
    _check(lib().fsc_embed_orthogonal(g.handle, int(l), int(t), int(every), int(seed) & (2**64 - 1), _ptr(out),
                                      C.byref(o), _stream(stream)), "fsc_embed_orthogonal")
    return out


def top_eigenvectors(g: Graph, l: int, t: int, seed: int, every: int = 4, out=None, threads_per_row: int = 0,
                     events=None, stream=None):
    """fsc_top_eigenvectors: Ritz pairs of M from orthogonal iteration.  Returns (values (l,) numpy,
    embedding n x pad_l(l) = D^-1/2 [Ritz vectors])."""
    torch = _torch()
    if out is None:
        out = torch.empty((g.n, pad_l(l)), dtype=torch.float32, device=g.device)
    _require_cuda(out, torch.float32, "out")
    vals = (C.c_double * int(l))()
    o = _opts(False, threads_per_row, events)
    _check(lib().fsc_top_eigenvectors(g.handle, int(l), int(t), int(every), int(seed) & (2**64 - 1), _ptr(out), vals,
                                      C.byref(o), _stream(stream)), "fsc_top_eigenvectors")
    import numpy as _np
    return _np.array(vals[:]), out


def kmeans_best(emb, l: int, k: int, seed: int, n_init: int, max_iter: int = 100, labels=None,
                want_centroids: bool = False, want_seeds: bool = False, stream=None):
    """fsc_kmeans_best: the lowest-inertia run of n_init restarts (seeds seed .. seed+n_init-1).
    Returns (labels, stats, centroids, seeds, best_run)."""
    torch = _torch()
    _require_cuda(emb, torch.float32, "emb")
    n, ld = emb.shape
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=emb.device)
    cen = torch.empty((k, l), dtype=torch.float64, device=emb.device) if want_centroids else None
    sd = torch.empty(k, dtype=torch.int64, device=emb.device) if want_seeds else None
    st = KmeansStats()
    run = C.c_int(-1)
    _check(lib().fsc_kmeans_best(_ptr(emb), n, int(l), int(ld), int(k), int(seed) & (2**64 - 1), int(n_init),
                                 int(max_iter), _ptr(labels), _ptr(cen), _ptr(sd), C.byref(st), C.byref(run),
                                 _stream(stream)), "fsc_kmeans_best")
    return labels, st.as_dict(), cen, sd, run.value


def partition_scores(labels_a, labels_b, ka: int, kb: int, stream=None):
    """fsc_partition_scores: (ARI, NMI) of two int32 CUDA labelings with values in [0, ka), [0, kb)."""
    out = (C.c_double * 2)()
    _check(lib().fsc_partition_scores(_ptr(labels_a), _ptr(labels_b), int(labels_a.numel()), int(ka), int(kb), out,
                                      _stream(stream)), "fsc_partition_scores")
    return float(out[0]), float(out[1])


def cluster(g: Graph, k: int, l: int, t: int, seed: int, store: int = F32, max_iter: int = 100, labels=None,
            rescale: bool = False, threads_per_row: int = 0, events=None, stream=None):
    """fsc_cluster (Algorithm 2 end to end).  Returns (labels, stats)."""
    torch = _torch()
    if labels is None:
        labels = torch.empty(g.n, dtype=torch.int32, device=g.device)
    st = KmeansStats()
    o = _opts(rescale, threads_per_row, events)
    _check(lib().fsc_cluster(g.handle, int(k), int(l), int(t), int(seed) & (2**64 - 1), int(store), int(max_iter),
                             _ptr(labels), C.byref(st), C.byref(o), _stream(stream)), "fsc_cluster")
    return labels, st.as_dict()


def autotune(g: Graph, l: int, store: int = F32, stream=None):
    """fsc_autotune: returns (best lanes per row, microseconds per power step)."""
    best, us = C.c_int(), C.c_float()
    _check(lib().fsc_autotune(g.handle, int(l), int(store), C.byref(best), C.byref(us), _stream(stream)),
           "fsc_autotune")
    return best.value, us.value


class Batch:
    """A batched clustering plan over the disjoint union of many graphs (fsc_batch_create).

    ``row_ptr``/``col`` (and ``w``) are the union CSR on the device with global vertex ids;
    ``vertex_offset`` (host, int64, G+1) delimits the graphs; ``k``, ``l``, ``t``, ``seed`` are
    per-graph host arrays (``l``/``t`` may be None for the defaults).  ``run()`` replays the
    captured CUDA graph; ``labels`` (device, int32) receives local cluster ids.
    """

    def __init__(self, vertex_offset, row_ptr, col, k, seed, w=None, l=None, t=None, store: int = F32,
                 max_iter: int = 100, autotune: bool = False, validate_symmetry: bool = False, stream=None):
        import numpy as np
        torch = _torch()
        _require_cuda(row_ptr, torch.int64, "row_ptr")
        _require_cuda(col, torch.int32, "col")
        if w is not None:
            _require_cuda(w, torch.float32, "w")
        self._host = {
            "voff": np.ascontiguousarray(vertex_offset, dtype=np.int64),
            "k": np.ascontiguousarray(k, dtype=np.int32),
            "seed": np.ascontiguousarray(seed, dtype=np.uint64),
            "l": None if l is None else np.ascontiguousarray(l, dtype=np.int32),
            "t": None if t is None else np.ascontiguousarray(t, dtype=np.int32),
        }
        self.num_graphs = len(self._host["k"])
        self.row_ptr, self.col, self.w = row_ptr, col, w
        nv = int(self._host["voff"][-1])
        self.labels = torch.empty(nv, dtype=torch.int32, device=row_ptr.device)
        d = BatchDesc()
        d.num_graphs = self.num_graphs
        d.vertex_offset = self._host["voff"].ctypes.data
        d.row_ptr = row_ptr.data_ptr()
        d.col_idx = col.data_ptr()
        d.w = None if w is None else w.data_ptr()
        d.k = self._host["k"].ctypes.data
        d.l = None if self._host["l"] is None else self._host["l"].ctypes.data
        d.t = None if self._host["t"] is None else self._host["t"].ctypes.data
        d.seed = self._host["seed"].ctypes.data
        d.labels = self.labels.data_ptr()
        d.store = int(store)
        d.max_iter = int(max_iter)
        d.flags = (BATCH_AUTOTUNE if autotune else 0) | (VALIDATE_SYMMETRY if validate_symmetry else 0)
        h = C.c_void_p()
        _check(lib().fsc_batch_create(C.byref(d), _stream(stream), C.byref(h)), "fsc_batch_create")
        self.handle = h

    def run(self, stream=None):
        _check(lib().fsc_batch_run(self.handle, _stream(stream)), "fsc_batch_run")
        return self.labels

    def results(self, stream=None):
        """(stats list, k-means++ picks per graph, centroids per graph) after a run (synchronises)."""
        import numpy as np
        G = self.num_graphs
        st = (KmeansStats * G)()
        k = self._host["k"]
        total_k = int(k.sum())
        seeds = np.zeros(total_k, dtype=np.int64)
        ls = self._host["l"]
        if ls is None or (ls == 0).any():
            ls = np.array([default_params(int(self._host["voff"][g + 1] - self._host["voff"][g]), int(k[g]))[0]
                           if ls is None or ls[g] == 0 else int(ls[g]) for g in range(G)], dtype=np.int64)
        cents = np.zeros(int((k.astype(np.int64) * ls).sum()), dtype=np.float64)
        _check(lib().fsc_batch_results(self.handle, C.cast(st, C.c_void_p), seeds.ctypes.data, cents.ctypes.data,
                                       _stream(stream)), "fsc_batch_results")
        so = co = 0
        seed_list, cent_list = [], []
        for g in range(G):
            seed_list.append(seeds[so:so + k[g]])
            cent_list.append(cents[co:co + k[g] * ls[g]].reshape(k[g], ls[g]))
            so += k[g]
            co += k[g] * ls[g]
        return [s.as_dict() for s in st], seed_list, cent_list

    def embedding(self, g: int, n: int, l: int, stream=None):
        """Graph g's float32 embedding (n x pad_l(l)) from the last run (device tensor)."""
        torch = _torch()
        out = torch.empty((n, pad_l(l)), dtype=torch.float32, device=self.row_ptr.device)
        _check(lib().fsc_batch_embedding(self.handle, int(g), _ptr(out), _stream(stream)), "fsc_batch_embedding")
        return out

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().fsc_batch_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NPARAM = 5833
FILTER_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "filter", "mlp_weights.npz")


def load_filter_params(path: str | None = None, device="cuda"):
    """The trained filter MLP parameters (5833 float32) as a device tensor."""
    import numpy as np
    torch = _torch()
    p = np.load(path or FILTER_WEIGHTS)["params"].astype(np.float32)
    assert p.size == NPARAM
    return torch.as_tensor(p, device=device)


def filter_embed(g: Graph, l: int, k: int, seed: int, params=None, coeffs=None, store: int = F32, out=None,
                 threads_per_row: int = 0, events=None, energy=None, stream=None):
    """fsc_filter_embed: returns (embedding n x pad_l(l), features (16), coefficients (9)) device tensors.
    ``energy`` (optional float64 CUDA tensor of one element) receives ||p(M) X||^2 (x-space)."""
    torch = _torch()
    dev = g.device
    if out is None:
        out = torch.empty((g.n, pad_l(l)), dtype=torch.float32, device=dev)
    feats = torch.empty(16, dtype=torch.float32, device=dev)
    cf = torch.empty(9, dtype=torch.float32, device=dev)
    o = _opts(False, threads_per_row, events)
    _check(lib().fsc_filter_embed(g.handle, int(l), int(k), int(seed) & (2**64 - 1), int(store), _ptr(params),
                                  _ptr(coeffs), _ptr(out), _ptr(feats), _ptr(cf), _ptr(energy), C.byref(o),
                                  _stream(stream)),
           "fsc_filter_embed")
    return out, feats, cf


def cluster_filtered(g: Graph, k: int, l: int, seed: int, params, store: int = F32, max_iter: int = 100,
                     labels=None, threads_per_row: int = 0, events=None, fallback: bool = True, stream=None):
    """fsc_cluster_filtered: Algorithm 2 with the learned filter in place of M^t.  Returns (labels, stats);
    stats also holds the guard's report (filter_energy_ratio, filter_threshold, fallback, fallback_t)."""
    torch = _torch()
    if labels is None:
        labels = torch.empty(g.n, dtype=torch.int32, device=g.device)
    st = KmeansStats()
    rep = FilterReport()
    o = _opts(False, threads_per_row, events)
    if not fallback:
        o.flags |= FILTER_NO_FALLBACK
    _check(lib().fsc_cluster_filtered(g.handle, int(k), int(l), int(seed) & (2**64 - 1), int(store), _ptr(params),
                                      int(max_iter), _ptr(labels), C.byref(st), C.byref(rep), C.byref(o),
                                      _stream(stream)),
           "fsc_cluster_filtered")
    out = st.as_dict()
    out.update(filter_energy_ratio=rep.energy_ratio, filter_threshold=rep.threshold, fallback=rep.fallback,
               fallback_t=rep.fallback_t)
    return labels, out


def mlp_forward(params, feats, stream=None):
    """fsc_mlp_forward: coefficients (B x 9) of features (B x 16)."""
    torch = _torch()
    out = torch.empty((feats.shape[0], 9), dtype=torch.float32, device=feats.device)
    _check(lib().fsc_mlp_forward(_ptr(params), _ptr(feats), int(feats.shape[0]), _ptr(out), _stream(stream)),
           "fsc_mlp_forward")
    return out


def mlp_train_step(params, grad, m, v, step, lr, feats, Gn, bn, weight_decay=0.0, loss=None, apply_update=True,
                   stream=None):
    """fsc_mlp_train_step (see the header): one gradient accumulation and optional Adam step."""
    _check(lib().fsc_mlp_train_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr),
                                    float(weight_decay), _ptr(feats), _ptr(Gn), _ptr(bn), int(feats.shape[0]),
                                    _ptr(loss), 1 if apply_update else 0, _stream(stream)), "fsc_mlp_train_step")
