"""Python binding of libmrq, the GB300 (sm_103a) implementation of MRQ
(projection + quantization approximate k-NN, arXiv 2411.06158).

Argument marshalling only: every step of index construction and search runs
in the CUDA library declared in ``include/mrq.h``; the functions below have the
same names as the C entry points.  Arrays may be numpy arrays (host) or torch
CUDA tensors (device); results come back in the same kind of memory as the
queries.  Importing this module fails loudly if ``libmrq.so`` is missing (run
``python -c "import __graft_entry__ as g; g.build()"`` first).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmrq.so")

MRQ_OK = 0
MRQ_EINVAL, MRQ_ENOMEM, MRQ_ECUDA, MRQ_EFORMAT, MRQ_EIO, MRQ_ETIMEDOUT = -1, -2, -3, -4, -5, -6
MODE_MRQ, MODE_MRQ_PLUS, MODE_SQ8, MODE_PQ = 0, 1, 2, 3
PREC_FP32, PREC_BF16, PREC_BF16X3, PREC_FP8 = 0, 1, 2, 3
SCAN_PAIRS, SCAN_BATCHED, SCAN_AUTO, SCAN_BATCHED_TC = 0, 1, 2, 3

EXPORTS = [
    "mrq_build_opts_default", "mrq_search_opts_default", "mrq_build", "mrq_search",
    "mrq_estimate", "mrq_project", "mrq_project_noalloc", "mrq_autotune", "mrq_last_search_stats", "mrq_last_search_profile",
    "mrq_save", "mrq_load",
    "mrq_index_info", "mrq_index_export", "mrq_free", "mrq_last_error",
    "mrq_server_opts_default", "mrq_server_start", "mrq_submit", "mrq_submit_many", "mrq_poll",
    "mrq_poll_many", "mrq_poll_completed", "mrq_server_stats", "mrq_server_reset_stats",
    "mrq_server_stop", "mrq_shard_plan", "mrq_index_shard", "mrq_merge_topk", "mrq_pq_train",
    "mrq_last_search_redo",
]


class MRQError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mrq error {code}: {msg}")
        self.code = code


class BuildOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("kmeans_iters", C.c_int),
                ("init_centroids", C.c_void_p), ("init_ids", C.c_void_p),
                ("rotation_gauss", C.c_void_p), ("auto_d_variance", C.c_double),
                ("pca_rows", C.c_void_p), ("pca_n", C.c_int64)]


class SearchOpts(C.Structure):
    _fields_ = [("eps0", C.c_float), ("m", C.c_float), ("mode", C.c_int),
                ("precision", C.c_int), ("query_bits", C.c_int), ("batched", C.c_int),
                ("profile", C.c_int), ("graph", C.c_int), ("refine", C.c_int),
                ("rerank", C.c_int), ("cuda_stream", C.c_void_p),
                ("survivor_region", C.c_int64)]


class ServerOpts(C.Structure):
    _fields_ = [("mem_budget", C.c_size_t), ("max_batch", C.c_int), ("max_inflight", C.c_int),
                ("max_wait_us", C.c_int), ("max_k", C.c_int), ("search", SearchOpts)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("batches", C.c_int64), ("pending", C.c_int64),
                ("p50_us", C.c_double), ("p99_us", C.c_double), ("max_us", C.c_double),
                ("qps", C.c_double)]


class TuneResult(C.Structure):
    _fields_ = [("scan", C.c_int), ("chunk", C.c_int), ("group", C.c_int), ("ms", C.c_double),
                ("ms_default", C.c_double), ("n_tried", C.c_int), ("consistent", C.c_int)]


class IndexInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("D", C.c_int), ("d", C.c_int), ("bits", C.c_int),
                ("nlist", C.c_int), ("max_list", C.c_int64), ("device_bytes", C.c_int64),
                ("pq_M", C.c_int), ("pq_K", C.c_int)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libmrq.so not built at {path}; call __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    lib.mrq_build_opts_default.argtypes = [C.POINTER(BuildOpts)]
    lib.mrq_search_opts_default.argtypes = [C.POINTER(SearchOpts)]
    lib.mrq_build.argtypes = [vp, i64, i32, i32, i32, i32, C.POINTER(BuildOpts), C.POINTER(vp)]
    lib.mrq_search.argtypes = [vp, vp, i64, i32, i32, C.POINTER(SearchOpts), vp, vp]
    lib.mrq_estimate.argtypes = [vp, vp, i32, C.POINTER(SearchOpts), vp, vp, vp, vp, vp]
    lib.mrq_project.argtypes = [vp, vp, i64, C.POINTER(SearchOpts), vp]
    lib.mrq_project_noalloc.argtypes = [vp, vp, i64, C.POINTER(SearchOpts), vp]
    lib.mrq_autotune.argtypes = [vp, vp, i64, i32, i32, C.POINTER(SearchOpts), C.POINTER(TuneResult)]
    lib.mrq_last_search_stats.argtypes = [vp, i64, vp, vp, vp]
    lib.mrq_last_search_profile.argtypes = [vp, vp, vp]
    lib.mrq_save.argtypes = [vp, C.c_char_p]
    lib.mrq_load.argtypes = [C.c_char_p, C.POINTER(vp)]
    lib.mrq_index_info.argtypes = [vp, C.POINTER(IndexInfo)]
    lib.mrq_index_export.argtypes = [vp, C.c_char_p, vp, C.c_size_t]
    lib.mrq_free.argtypes = [vp]
    lib.mrq_free.restype = None
    lib.mrq_server_opts_default.argtypes = [C.POINTER(ServerOpts)]
    lib.mrq_server_opts_default.restype = None
    lib.mrq_server_start.argtypes = [vp, C.POINTER(ServerOpts), C.POINTER(vp)]
    lib.mrq_submit.argtypes = [vp, vp, i32, i32, vp]
    lib.mrq_submit_many.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.mrq_poll.argtypes = [vp, C.c_uint64, vp, vp, i32]
    lib.mrq_poll_many.argtypes = [vp, i64, vp, i32, vp, vp, vp]
    lib.mrq_poll_completed.argtypes = [vp, i64, i32, vp, vp, vp, vp]
    lib.mrq_server_stats.argtypes = [vp, C.POINTER(ServerStats)]
    lib.mrq_server_reset_stats.argtypes = [vp]
    lib.mrq_server_stop.argtypes = [vp]
    lib.mrq_pq_train.argtypes = [vp, i32, i32, i32, i32, vp, C.c_uint64]
    lib.mrq_last_search_redo.argtypes = [vp, vp]
    lib.mrq_shard_plan.argtypes = [vp, i32, i32, vp]
    lib.mrq_index_shard.argtypes = [vp, i32, i32, C.POINTER(vp)]
    lib.mrq_merge_topk.argtypes = [vp, vp, i32, i64, i32, vp, vp, vp]
    lib.mrq_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("mrq_free", "mrq_last_error", "mrq_build_opts_default",
                        "mrq_search_opts_default", "mrq_server_opts_default"):
            getattr(lib, name).restype = C.c_int
    lib.mrq_poll_completed.restype = C.c_int64
    return lib


_lib = load_library()


def _check(rc: int) -> None:
    if rc != MRQ_OK:
        raise MRQError(rc, _lib.mrq_last_error().decode(errors="replace"))


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Raw pointer of a C-contiguous numpy array or torch tensor."""
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_contiguous(), "tensor must be contiguous"
        return x.data_ptr()
    assert x.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return x.ctypes.data


def _f32(x):
    if _is_torch(x):
        import torch
        return x.to(torch.float32).contiguous()
    return np.ascontiguousarray(x, dtype=np.float32)


def mrq_build_opts(seed: int = 1, kmeans_iters: int = 20, init_centroids=None, init_ids=None,
                   rotation_gauss=None, auto_d_variance: float = 0.8, pca_rows=None):
    """Build options plus the arrays that must stay alive during the call."""
    o = BuildOpts()
    _lib.mrq_build_opts_default(C.byref(o))
    o.seed, o.kmeans_iters, o.auto_d_variance = seed, kmeans_iters, auto_d_variance
    keep = []
    if pca_rows is not None:
        a = np.ascontiguousarray(pca_rows, dtype=np.int64)
        keep.append(a)
        o.pca_rows, o.pca_n = a.ctypes.data, a.shape[0]
    if init_centroids is not None:
        a = np.ascontiguousarray(init_centroids, dtype=np.float32)
        keep.append(a)
        o.init_centroids = a.ctypes.data
    if init_ids is not None:
        a = np.ascontiguousarray(init_ids, dtype=np.int64)
        keep.append(a)
        o.init_ids = a.ctypes.data
    if rotation_gauss is not None:
        a = np.ascontiguousarray(rotation_gauss, dtype=np.float64)
        keep.append(a)
        o.rotation_gauss = a.ctypes.data
    return o, keep


def mrq_search_opts(eps0: float = 1.9, m: float = 4.0, mode: int = MODE_MRQ_PLUS,
                    precision: int = PREC_FP32, query_bits: int = 0, batched: int = 0,
                    profile: int = 0, graph: int = 0, stream=None, refine: int = 0,
                    rerank: int = 500, survivor_region: int = 0) -> SearchOpts:
    o = SearchOpts()
    _lib.mrq_search_opts_default(C.byref(o))
    o.eps0, o.m, o.mode, o.precision = eps0, m, mode, precision
    o.query_bits, o.batched, o.profile, o.graph = query_bits, batched, profile, graph
    o.refine, o.rerank, o.survivor_region = refine, rerank, survivor_region
    if stream is not None:
        o.cuda_stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return o


class Index:
    """Owning handle of an mrq_index (freed with mrq_free)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.mrq_free(self.handle)
            self.handle = C.c_void_p(None)

    def info(self) -> IndexInfo:
        return mrq_index_info(self)


def mrq_build(base, d: int, bits: int, nlist: int, opts=None) -> Index:
    base = _f32(base)
    n, D = base.shape
    o, keep = opts if isinstance(opts, tuple) else (opts, [])
    h = C.c_void_p()
    _check(_lib.mrq_build(_ptr(base), n, D, d, bits, nlist,
                          C.byref(o) if o is not None else None, C.byref(h)))
    return Index(h.value)


def _out_like(q, shape, kind):
    if _is_torch(q) and q.is_cuda:
        import torch
        return torch.empty(shape, dtype=kind[0], device=q.device)
    return np.empty(shape, dtype=kind[1])


def mrq_search(index: Index, queries, k: int, nprobe: int, opts: SearchOpts | None = None,
               out=None):
    """Return (ids int64 [nq, k], dists float32 [nq, k]) sorted by (dist, id)."""
    import_torch = _is_torch(queries)
    queries = _f32(queries)
    nq = queries.shape[0]
    if out is None:
        if import_torch:
            import torch
            ids = _out_like(queries, (nq, k), (torch.int64, np.int64))
            dists = _out_like(queries, (nq, k), (torch.float32, np.float32))
        else:
            ids = np.empty((nq, k), dtype=np.int64)
            dists = np.empty((nq, k), dtype=np.float32)
    else:
        ids, dists = out
    _check(_lib.mrq_search(index.handle, _ptr(queries), nq, k, nprobe,
                           C.byref(opts) if opts is not None else None, _ptr(ids), _ptr(dists)))
    return ids, dists


def mrq_estimate(index: Index, qp, list_id: int, opts: SearchOpts | None = None):
    """Per-candidate stage-1 values of one projected query against one list."""
    qp = np.ascontiguousarray(qp, dtype=np.float32)
    info = index.info()
    loff = mrq_index_export(index, "LOFF")
    sz = int(loff[list_id + 1] - loff[list_id])
    ip, dis, lb, ub = (np.zeros(sz, dtype=np.float32) for _ in range(4))
    idot = np.zeros(sz, dtype=np.int32)
    _check(_lib.mrq_estimate(index.handle, _ptr(qp), list_id,
                             C.byref(opts) if opts is not None else None,
                             _ptr(ip), _ptr(dis), _ptr(lb), _ptr(ub), _ptr(idot)))
    del info
    return dict(ip=ip, dis=dis, lb=lb, ub=ub, int_dot=idot)


def mrq_project(index: Index, queries, opts: SearchOpts | None = None):
    queries = _f32(queries)
    nq = queries.shape[0]
    D = index.info().D
    out = _out_like(queries, (nq, D), (__import__("torch").float32, np.float32)) \
        if _is_torch(queries) else np.empty((nq, D), dtype=np.float32)
    _check(_lib.mrq_project(index.handle, _ptr(queries), nq,
                            C.byref(opts) if opts is not None else None, _ptr(out)))
    return out


def mrq_project_noalloc(index: Index, queries, out, opts: SearchOpts | None = None):
    """mrq_project into a caller-owned device tensor `out` (nq x D float32) from
    device `queries`, through the entry point that allocates no device memory."""
    nq = queries.shape[0]
    _check(_lib.mrq_project_noalloc(index.handle, _ptr(queries), nq,
                                    C.byref(opts) if opts is not None else None, _ptr(out)))
    return out


def mrq_autotune(index: Index, queries, k: int, nprobe: int, opts: SearchOpts | None = None):
    """Time the scan decompositions on `queries` and record the fastest for
    (k, nprobe, opts.query_bits); searches with batched=SCAN_AUTO use it."""
    queries = _f32(queries)
    r = TuneResult()
    _check(_lib.mrq_autotune(index.handle, _ptr(queries), queries.shape[0], k, nprobe,
                             C.byref(opts) if opts is not None else None, C.byref(r)))
    return {f: getattr(r, f) for f, _ in TuneResult._fields_}


def mrq_last_search_stats(index: Index, nq: int):
    a, b, c = (np.zeros(nq, dtype=np.int64) for _ in range(3))
    _check(_lib.mrq_last_search_stats(index.handle, nq, _ptr(a), _ptr(b), _ptr(c)))
    return dict(n_cand=a, n_s1=b, n_exact=c)


STAGES = ["project", "qstats", "probe", "select", "scan", "tau_a", "stage2", "tau_b", "exact",
          "topk"]


def mrq_last_search_profile(index: Index):
    """(stage -> device milliseconds, kernel launches) of the last profiled search."""
    ms = np.zeros(len(STAGES), dtype=np.float64)
    n = np.zeros(1, dtype=np.int64)
    _check(_lib.mrq_last_search_profile(index.handle, _ptr(ms), _ptr(n)))
    return dict(zip(STAGES, ms.tolist())), int(n[0])


def mrq_save(index: Index, path: str) -> None:
    _check(_lib.mrq_save(index.handle, path.encode()))


def mrq_load(path: str) -> Index:
    h = C.c_void_p()
    _check(_lib.mrq_load(path.encode(), C.byref(h)))
    return Index(h.value)


def mrq_index_info(index: Index) -> IndexInfo:
    info = IndexInfo()
    _check(_lib.mrq_index_info(index.handle, C.byref(info)))
    return info


_FIELD_SHAPES = {
    "MU__": (np.float32, lambda i: (i.D,)), "LAM_": (np.float32, lambda i: (i.D,)),
    "W___": (np.float32, lambda i: (i.D, i.D)), "CENT": (np.float32, lambda i: (i.nlist, i.d)),
    "LOFF": (np.int64, lambda i: (i.nlist + 1,)), "IDS_": (np.int64, lambda i: (i.n,)),
    "CODE": (np.uint8, lambda i: (i.n, i.d)), "FADD": (np.float32, lambda i: (i.n,)),
    "FRES": (np.float32, lambda i: (i.n,)), "FERR": (np.float32, lambda i: (i.n,)),
    "XD__": (np.float32, lambda i: (i.n, i.d)), "XR__": (np.float32, lambda i: (i.n, i.D - i.d)),
    "XN2_": (np.float32, lambda i: (i.n,)),
    "FRE1": (np.float32, lambda i: (i.n,)), "FER1": (np.float32, lambda i: (i.n,)),
    "SQ8C": (np.uint8, lambda i: (i.n, i.d)), "SQ8L": (np.float32, lambda i: (i.d,)),
    "SQ8S": (np.float32, lambda i: (i.d,)),
    "PQR_": (np.float32, lambda i: (i.d, i.d)),
    "PQC_": (np.float32, lambda i: (i.pq_M, i.pq_K, i.d // max(i.pq_M, 1))),
    "PQK_": (np.uint8, lambda i: (i.n, i.pq_M)),
}


def mrq_index_export(index: Index, field: str) -> np.ndarray:
    info = index.info()
    dt, shp = _FIELD_SHAPES[field]
    out = np.empty(shp(info), dtype=dt)
    _check(_lib.mrq_index_export(index.handle, field.encode(), _ptr(out), out.nbytes))
    return out


def mrq_last_search_redo(index: Index) -> int:
    """Queries of the last search searched again with a larger survivor region."""
    n = np.zeros(1, dtype=np.int64)
    _check(_lib.mrq_last_search_redo(index.handle, _ptr(n)))
    return int(n[0])


def mrq_pq_train(index: Index, M: int, K: int = 16, opq_iters: int = 4, km_iters: int = 6,
                 init_rows=None, seed: int = 1) -> None:
    """Train the OPQ of MODE_PQ on the GPU (rows of the list-major x_d' as initial
    centroids: ``init_rows``, or K rows drawn from ``seed``)."""
    keep = None
    if init_rows is not None:
        keep = np.ascontiguousarray(init_rows, dtype=np.int64)
    _check(_lib.mrq_pq_train(index.handle, M, K, opq_iters, km_iters, _ptr(keep), seed))


def mrq_shard_plan(list_sizes, nshards: int) -> np.ndarray:
    """Shard of every IVF list under the library's partition plan (host only)."""
    sizes = np.ascontiguousarray(list_sizes, dtype=np.int64)
    owner = np.empty(sizes.shape[0], dtype=np.int32)
    _check(_lib.mrq_shard_plan(_ptr(sizes), sizes.shape[0], nshards, _ptr(owner)))
    return owner


def mrq_index_shard(index: Index, nshards: int, shard: int) -> Index:
    """The index of shard `shard` of `nshards` (every centroid, its own lists' members)."""
    h = C.c_void_p()
    _check(_lib.mrq_index_shard(index.handle, nshards, shard, C.byref(h)))
    return Index(h.value)


def mrq_merge_topk(ids, dists, k: int, out=None, stream=None):
    """Merge per-part answers: ids / dists are (nparts, nq, k), numpy arrays or CUDA
    tensors; returns (ids, dists) of shape (nq, k) in the same kind of memory."""
    nparts, nq = int(ids.shape[0]), int(ids.shape[1])
    if out is None:
        if _is_torch(ids):
            import torch
            out = (torch.empty((nq, k), dtype=torch.int64, device=ids.device),
                   torch.empty((nq, k), dtype=torch.float32, device=ids.device))
        else:
            out = (np.empty((nq, k), dtype=np.int64), np.empty((nq, k), dtype=np.float32))
    if not _is_torch(ids):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        dists = np.ascontiguousarray(dists, dtype=np.float32)
    st = None
    if stream is not None:
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(_lib.mrq_merge_topk(_ptr(ids), _ptr(dists), nparts, nq, k, st, _ptr(out[0]),
                               _ptr(out[1])))
    return out


def mrq_free(index: Index) -> None:
    index.__del__()


def mrq_last_error() -> str:
    return _lib.mrq_last_error().decode(errors="replace")


# ------------------------------------------------------------------ serving

class Server:
    """Owning handle of an mrq_server (continuous batching over one index)."""

    def __init__(self, index: Index, mem_budget: int | None = None, max_batch: int = 4096,
                 max_inflight: int = 4, max_wait_us: int = 300, max_k: int = 128,
                 search: SearchOpts | None = None):
        o = ServerOpts()
        _lib.mrq_server_opts_default(C.byref(o))
        if mem_budget is not None:
            o.mem_budget = mem_budget
        o.max_batch, o.max_inflight, o.max_wait_us, o.max_k = max_batch, max_inflight, max_wait_us, max_k
        if search is not None:
            o.search = search
        h = C.c_void_p()
        _check(_lib.mrq_server_start(index.handle, C.byref(o), C.byref(h)))
        self.index, self.handle, self.max_k, self.D = index, h, max_k, index.info().D

    def submit(self, query, k: int, nprobe: int) -> int:
        q = np.ascontiguousarray(query, dtype=np.float32)
        t = C.c_uint64()
        _check(_lib.mrq_submit(self.handle, _ptr(q), k, nprobe, C.byref(t)))
        return t.value

    def submit_many(self, queries, k, nprobe) -> np.ndarray:
        q = np.ascontiguousarray(queries, dtype=np.float32)
        n = q.shape[0]
        ks = np.ascontiguousarray(np.broadcast_to(k, (n,)), dtype=np.int32)
        ps = np.ascontiguousarray(np.broadcast_to(nprobe, (n,)), dtype=np.int32)
        t = np.empty(n, dtype=np.uint64)
        _check(_lib.mrq_submit_many(self.handle, n, _ptr(q), _ptr(ks), _ptr(ps), _ptr(t)))
        return t

    def poll(self, ticket: int, k: int, wait_ms: int = 0):
        """(ids, dists) when done, else None."""
        ids = np.empty(k, dtype=np.int64)
        d = np.empty(k, dtype=np.float32)
        rc = _lib.mrq_poll(self.handle, ticket, _ptr(ids), _ptr(d), wait_ms)
        if rc == 1:
            return None
        _check(rc)
        return ids, d

    def poll_many(self, tickets, kmax: int):
        t = np.ascontiguousarray(tickets, dtype=np.uint64)
        n = t.shape[0]
        ids = np.empty((n, kmax), dtype=np.int64)
        d = np.empty((n, kmax), dtype=np.float32)
        st = np.empty(n, dtype=np.int32)
        _check(_lib.mrq_poll_many(self.handle, n, _ptr(t), kmax, _ptr(ids), _ptr(d), _ptr(st)))
        return ids, d, st

    def poll_completed(self, max_n: int, kmax: int):
        """(tickets, ids, dists, status) of up to max_n completed requests, released."""
        t = np.empty(max_n, dtype=np.uint64)
        ids = np.empty((max_n, kmax), dtype=np.int64)
        d = np.empty((max_n, kmax), dtype=np.float32)
        st = np.empty(max_n, dtype=np.int32)
        n = _lib.mrq_poll_completed(self.handle, max_n, kmax, _ptr(t), _ptr(ids), _ptr(d), _ptr(st))
        if n < 0:
            _check(int(n))
        return t[:n], ids[:n], d[:n], st[:n]

    def stats(self) -> dict:
        s = ServerStats()
        _check(_lib.mrq_server_stats(self.handle, C.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def reset_stats(self) -> None:
        _check(_lib.mrq_server_reset_stats(self.handle))

    def stop(self) -> None:
        if self.handle is not None and self.handle.value:
            h, self.handle = self.handle, None
            _check(_lib.mrq_server_stop(h))

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def mrq_server_start(index: Index, **kw) -> Server:
    return Server(index, **kw)
