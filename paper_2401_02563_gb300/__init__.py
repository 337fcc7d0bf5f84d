"""Python binding of the GB300 temporal edge-map library (libkairos.so, C ABI in
include/kairos.h).

Argument marshalling only: every function below converts numpy arrays / torch tensors to
pointers and calls the C function of the same name; all query work happens in the
library's CUDA kernels.  There is no CPU fallback: if the library cannot be loaded, every
call raises.

Device memory and streams come from PyTorch: pass torch CUDA tensors as outputs, a
torch.cuda.Stream (or its handle) as the graph stream, and optionally let the library
allocate through torch's caching allocator.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

KAIROS_OK = 0
KAIROS_ERR_INVALID_ARG = 1
KAIROS_ERR_OOM = 2
KAIROS_ERR_CUDA = 3
KAIROS_ERR_OVERFLOW = 4
KAIROS_ERR_NOT_READY = 5
KAIROS_ERR_BUSY = 6
KAIROS_ERR_TIMEOUT = 7
KAIROS_ERR_INTERNAL = 8
KAIROS_UNREACHED = 0xFFFFFFFF
KAIROS_TIME_MAX = 0xFFFFFFFE
KAIROS_NO_INDEX = 0xFFFFFFFF
KAIROS_EA = 0
KAIROS_LD = 1

_P = ctypes.c_void_p


class kairos_edge_list(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_edges", ctypes.c_int64), ("src", _P), ("dst", _P),
                ("t_dep", _P), ("lambda_", _P), ("lambda_bits", ctypes.c_int32), ("on_device", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class kairos_graph_opts(ctypes.Structure):
    _fields_ = [("stream", _P), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", _P),
                ("skip_reverse", ctypes.c_int32)]


class kairos_query(ctypes.Structure):
    _fields_ = [("vertex", ctypes.c_int32), ("ta", ctypes.c_uint32), ("tw", ctypes.c_uint32),
                ("kind", ctypes.c_uint8), ("strict", ctypes.c_uint8), ("reserved", ctypes.c_uint16)]


class kairos_query_stats(ctypes.Structure):
    _fields_ = [("relaxed_edges", ctypes.c_uint64), ("scanned_edges", ctypes.c_uint64),
                ("rounds", ctypes.c_uint32), ("reached", ctypes.c_uint32)]


class kairos_tuning(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("warp_max_edges", ctypes.c_int32),
                ("chunk_edges", ctypes.c_int32), ("dense_div", ctypes.c_int32), ("relax_mode", ctypes.c_int32),
                ("concurrent", ctypes.c_int32), ("block_edges", ctypes.c_int32),
                ("select_permille", ctypes.c_int32)]


class kairos_graph_info(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_edges", ctypes.c_int64), ("lambda_bits", ctypes.c_int32),
                ("index_threshold", ctypes.c_uint32), ("indexed_vertices", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("build_ms", ctypes.c_double), ("index_ms", ctypes.c_double),
                ("graph_launches", ctypes.c_int64)]


class kairos_serve_opts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("queue_capacity", ctypes.c_int32), ("reserve_bytes", ctypes.c_int64),
                ("rounds_per_slice", ctypes.c_int32)]


class kairos_result_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reached", ctypes.c_uint32), ("relaxed_edges", ctypes.c_uint64),
                ("checksum", ctypes.c_uint64), ("latency_ms", ctypes.c_double)]


class kairos_fastest_stats(ctypes.Structure):
    _fields_ = [("start_times", ctypes.c_uint64), ("launches", ctypes.c_uint64), ("relaxed_edges", ctypes.c_uint64)]


class kairos_duration_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint64), ("examined_edges", ctypes.c_uint64)]


# Every function the header declares, with its ctypes signature.
SIGNATURES = {
    "kairos_graph_build": (ctypes.c_int, [ctypes.POINTER(kairos_edge_list), ctypes.POINTER(kairos_graph_opts),
                                          ctypes.POINTER(_P)]),
    "kairos_index_build": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "kairos_graph_free": (None, [_P]),
    "kairos_graph_get_info": (ctypes.c_int, [_P, ctypes.POINTER(kairos_graph_info)]),
    "kairos_earliest_arrival": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, _P]),
    "kairos_latest_departure": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, _P]),
    "kairos_batch_query": (ctypes.c_int, [_P, ctypes.POINTER(kairos_query), ctypes.c_int32, _P,
                                          ctypes.POINTER(kairos_query_stats)]),
    "kairos_fastest_path": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32, _P,
                                           ctypes.POINTER(kairos_fastest_stats)]),
    "kairos_shortest_duration": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                                ctypes.c_int32, _P, ctypes.POINTER(kairos_duration_stats)]),
    "kairos_temporal_bfs": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_int32, _P, ctypes.POINTER(kairos_duration_stats)]),
    "kairos_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(kairos_tuning)]),
    "kairos_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(kairos_tuning)]),
    "kairos_autotune": (ctypes.c_int, [_P, ctypes.POINTER(kairos_query), ctypes.c_int32,
                                       ctypes.POINTER(kairos_tuning)]),
    "kairos_autotune_from": (ctypes.c_int, [_P, ctypes.POINTER(kairos_query), ctypes.c_int32, ctypes.c_int32,
                                            ctypes.POINTER(kairos_tuning)]),
    "kairos_autotune_index": (ctypes.c_int, [_P, ctypes.POINTER(kairos_query), ctypes.c_int32, _P, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_uint32), _P]),
    "kairos_serve_create": (ctypes.c_int, [_P, ctypes.POINTER(kairos_serve_opts), ctypes.POINTER(_P)]),
    "kairos_serve_submit": (ctypes.c_int, [_P, ctypes.POINTER(kairos_query), _P, ctypes.POINTER(ctypes.c_uint64)]),
    "kairos_serve_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(kairos_result_info)]),
    "kairos_serve_destroy": (None, [_P]),
    "kairos_last_error": (ctypes.c_char_p, []),
    "kairos_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "kairos_last_kernel_ms": (ctypes.c_double, [_P]),
    "kairos_last_round_profile": (ctypes.c_int32, [_P, ctypes.c_int32, _P, _P, _P]),
    "kairos_last_phase_cycles": (ctypes.c_int32, [_P, _P]),
    "kairos_earliest_arrival_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, _P]),
    "kairos_last_stream_profile": (ctypes.c_int32, [_P, _P]),
    "kairos_temporal_cc": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint32, _P]),
    "kairos_selectivity_build": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "kairos_selectivity_estimate": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_uint32,
                                                   ctypes.c_uint32, ctypes.c_uint32, _P, _P]),
    "kairos_selectivity_histogram": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "kairos_router_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    "kairos_router_submit": (ctypes.c_int, [_P, ctypes.POINTER(kairos_query), _P, ctypes.POINTER(ctypes.c_uint64)]),
    "kairos_router_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(kairos_result_info)]),
    "kairos_router_replica_counts": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32]),
    "kairos_router_destroy": (None, [_P]),
}


def graph_fingerprint(n_vertices, src, dst, t_dep, lam, samples=4096) -> str:
    """A short hash of a graph's size and of evenly spaced samples of its edge arrays (host
    arrays or torch tensors): equal graphs agree; different ones almost surely differ."""
    import hashlib
    h = hashlib.sha256()
    m = int(src.shape[0])
    h.update(f"{int(n_vertices)}:{m}".encode())
    if m == 0:
        return h.hexdigest()[:24]
    idx = np.unique(np.linspace(0, m - 1, num=min(samples, m)).astype(np.int64))
    try:
        for a in (src, dst, t_dep, lam):
            if isinstance(a, np.ndarray):
                part = np.ascontiguousarray(a[idx])
            else:  # a torch tensor: gather through a signed view (unsigned types index poorly)
                import torch
                v = a.view(torch.int16) if a.element_size() == 2 else a.view(torch.int32)
                part = v[torch.as_tensor(idx, device=a.device)].cpu().numpy()
            h.update(f"{part.dtype.itemsize}".encode())
            h.update(part.tobytes())
    except Exception:  # the fingerprint only keys the autotune cache: never fail a build over it
        h.update(b"unsampled")
    return h.hexdigest()[:24]


_lib_digest = None


def _library_digest() -> str:
    global _lib_digest
    if _lib_digest is None:
        import hashlib
        with open(library_path(), "rb") as fh:
            _lib_digest = hashlib.sha256(fh.read()).hexdigest()[:16]
    return _lib_digest


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def autotune_cache_key(graph, sample) -> str:
    import hashlib
    qarr, k = make_queries(sample)
    qh = hashlib.sha256(ctypes.string_at(ctypes.addressof(qarr), ctypes.sizeof(kairos_query) * k)).hexdigest()[:16]
    return "|".join([graph.fingerprint, str(graph.theta), qh, _device_name(), _library_digest()])


def _read_cache(path) -> dict:
    import json
    try:
        with open(path) as fh:
            return json.load(fh)
    except (FileNotFoundError, ValueError):
        return {}


def _write_cache(path, table) -> None:
    import json
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


class KairosError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libkairos.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libkairos.so is not built; run __graft_entry__.build()")
            L = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(st: int, where: str):
    if st != KAIROS_OK:
        raise KairosError(st, where, lib().kairos_last_error().decode())


def _ptr(x):
    """Pointer of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _on_device(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def _nbytes(x) -> int:
    if isinstance(x, np.ndarray):
        return x.nbytes
    return x.numel() * x.element_size()


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class TorchAllocator:
    """Device allocator hooks that route the library's allocations through PyTorch's
    caching allocator on the current device."""

    def __init__(self):
        import torch
        self._torch = torch
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:
            return None

    def _free(self, ptr, ctx):
        if ptr:
            self._torch.cuda.caching_allocator_delete(int(ptr))


# ---- the C functions, one wrapper each ------------------------------------------------

def kairos_graph_build(n_vertices, src, dst, t_dep, lam, stream=None, allocator=None, skip_reverse=False):
    """Build a device graph from four equal-length arrays (numpy host arrays or torch
    tensors on the current CUDA device).  lam is uint16 or uint32.  Returns the handle."""
    m = int(src.shape[0])
    for a in (dst, t_dep, lam):
        if int(a.shape[0]) != m:
            raise ValueError("edge arrays differ in length")
    lam_bits = 8 * (lam.itemsize if isinstance(lam, np.ndarray) else lam.element_size())
    if lam_bits not in (16, 32):
        raise ValueError("lambda must be 16- or 32-bit")
    for a, sz in ((src, 4), (dst, 4), (t_dep, 4)):
        if (a.itemsize if isinstance(a, np.ndarray) else a.element_size()) != sz:
            raise ValueError("src, dst and t_dep must be 32-bit")
    dev = [_on_device(a) for a in (src, dst, t_dep, lam)]
    if any(dev) and not all(dev):
        raise ValueError("edge arrays must all be host or all be device")
    el = kairos_edge_list(int(n_vertices), m, _ptr(src), _ptr(dst), _ptr(t_dep), _ptr(lam), lam_bits,
                          1 if all(dev) else 0)
    opts = kairos_graph_opts()
    opts.stream = _stream_handle(stream)
    if allocator is not None:
        opts.alloc = allocator.alloc
        opts.free = allocator.free
    opts.skip_reverse = 1 if skip_reverse else 0
    h = _P()
    _check(lib().kairos_graph_build(ctypes.byref(el), ctypes.byref(opts), ctypes.byref(h)), "kairos_graph_build")
    return h


def kairos_index_build(g, threshold: int):
    _check(lib().kairos_index_build(g, int(threshold) & 0xFFFFFFFF), "kairos_index_build")


def kairos_graph_free(g):
    lib().kairos_graph_free(g)


def kairos_graph_get_info(g) -> kairos_graph_info:
    info = kairos_graph_info()
    _check(lib().kairos_graph_get_info(g, ctypes.byref(info)), "kairos_graph_get_info")
    return info


def _check_out(out, n, rows=1):
    if out is None or _nbytes(out) < 4 * n * rows:
        raise ValueError(f"out must hold {rows} x {n} uint32 labels")


def kairos_earliest_arrival(g, n, src, ta, tw, out):
    _check_out(out, n)
    _check(lib().kairos_earliest_arrival(g, int(src), int(ta), int(tw), _ptr(out)), "kairos_earliest_arrival")
    return out


def kairos_latest_departure(g, n, dst, ta, tw, out):
    _check_out(out, n)
    _check(lib().kairos_latest_departure(g, int(dst), int(ta), int(tw), _ptr(out)), "kairos_latest_departure")
    return out


def kairos_fastest_path(g, n, src, ta, tw, out, strict=0, want_stats=False):
    """Fastest-path durations from src into out (uint32[n], host or device); returns the
    kairos_fastest_stats when want_stats (relaxations are then counted)."""
    _check_out(out, n)
    st = kairos_fastest_stats() if want_stats else None
    _check(lib().kairos_fastest_path(g, int(src), int(ta), int(tw), int(strict), _ptr(out),
                                     ctypes.byref(st) if want_stats else None), "kairos_fastest_path")
    return st


def kairos_shortest_duration(g, n, src, ta, tw, out, strict=0):
    """Shortest-duration labels from src into out (uint32[n], host or device); returns the
    kairos_duration_stats."""
    _check_out(out, n)
    st = kairos_duration_stats()
    _check(lib().kairos_shortest_duration(g, int(src), int(ta), int(tw), int(strict), _ptr(out), ctypes.byref(st)),
           "kairos_shortest_duration")
    return st


def kairos_temporal_bfs(g, n, src, ta, tw, out, strict=0):
    """Temporal BFS levels (least number of edges) from src into out; returns the stats."""
    _check_out(out, n)
    st = kairos_duration_stats()
    _check(lib().kairos_temporal_bfs(g, int(src), int(ta), int(tw), int(strict), _ptr(out), ctypes.byref(st)),
           "kairos_temporal_bfs")
    return st


def kairos_earliest_arrival_noalloc(g, n, src, ta, tw, out):
    """Earliest arrival that allocates no device memory; out must be a CUDA tensor."""
    _check_out(out, n)
    _check(lib().kairos_earliest_arrival_noalloc(g, int(src), int(ta), int(tw), _ptr(out)),
           "kairos_earliest_arrival_noalloc")
    return out


def make_queries(queries) -> ctypes.Array:
    """queries: iterable of (kind, vertex, ta, tw[, strict]) or objects with those fields."""
    qs = list(queries)
    arr = (kairos_query * max(len(qs), 1))()
    for i, q in enumerate(qs):
        if isinstance(q, tuple):
            kind, v, ta, tw = q[:4]
            strict = q[4] if len(q) > 4 else 0
        else:
            kind, v, ta, tw, strict = q.kind, q.vertex, q.ta, q.tw, getattr(q, "strict", 0)
        arr[i] = kairos_query(int(v), int(ta), int(tw), int(kind), int(strict), 0)
    return arr, len(qs)


def kairos_batch_query(g, n, queries, out, want_stats=True):
    """out: [len(queries)][n] uint32 labels (numpy or torch, host or device).  Returns the
    per-query kairos_query_stats list (or None)."""
    qarr, k = make_queries(queries)
    _check_out(out, n, k)
    stats = (kairos_query_stats * max(k, 1))() if want_stats else None
    _check(lib().kairos_batch_query(g, qarr, k, _ptr(out), stats), "kairos_batch_query")
    return list(stats)[:k] if want_stats else None


def kairos_get_tuning(g) -> kairos_tuning:
    t = kairos_tuning()
    _check(lib().kairos_get_tuning(g, ctypes.byref(t)), "kairos_get_tuning")
    return t


def kairos_set_tuning(g, **fields):
    t = kairos_get_tuning(g)
    for k, v in fields.items():
        setattr(t, k, int(v))
    _check(lib().kairos_set_tuning(g, ctypes.byref(t)), "kairos_set_tuning")
    return t


def kairos_autotune(g, sample, min_lanes=1) -> kairos_tuning:
    qarr, k = make_queries(sample)
    best = kairos_tuning()
    _check(lib().kairos_autotune_from(g, qarr, k, int(min_lanes), ctypes.byref(best)), "kairos_autotune")
    return best


def kairos_autotune_index(g, sample, thetas):
    """Pick the index threshold among `thetas` by timing `sample`; returns (best, {theta: ms})."""
    qarr, k = make_queries(sample)
    th = np.ascontiguousarray(np.array([int(x) & 0xFFFFFFFF for x in thetas], np.uint32))
    ms = np.zeros(len(th), np.float64)
    best = ctypes.c_uint32(0)
    _check(lib().kairos_autotune_index(g, qarr, k, th.ctypes.data, len(th), ctypes.byref(best), ms.ctypes.data),
           "kairos_autotune_index")
    return int(best.value), dict(zip(th.tolist(), ms.tolist()))


def kairos_serve_create(g, max_slots=0, queue_capacity=0, reserve_bytes=0, rounds_per_slice=0):
    opts = kairos_serve_opts(int(max_slots), int(queue_capacity), int(reserve_bytes), int(rounds_per_slice))
    h = _P()
    _check(lib().kairos_serve_create(g, ctypes.byref(opts), ctypes.byref(h)), "kairos_serve_create")
    return h


def kairos_serve_submit(s, query, out) -> int:
    """Returns the ticket; raises KairosError (status BUSY) when the queue is full."""
    qarr, _ = make_queries([query])
    ticket = ctypes.c_uint64(0)
    _check(lib().kairos_serve_submit(s, qarr, _ptr(out), ctypes.byref(ticket)), "kairos_serve_submit")
    return int(ticket.value)


def kairos_serve_poll(s, ticket, timeout_us=-1):
    """Returns kairos_result_info, or None while the query is still running."""
    info = kairos_result_info()
    st = lib().kairos_serve_poll(s, int(ticket), int(timeout_us), ctypes.byref(info))
    if st == KAIROS_ERR_NOT_READY:
        return None
    _check(st, "kairos_serve_poll")
    return info


def kairos_serve_destroy(s):
    lib().kairos_serve_destroy(s)


def kairos_temporal_cc(g, n, ta, tw, out):
    """Component labels (smallest vertex id) of the window's snapshot into out (n labels)."""
    _check_out(out, n)
    _check(lib().kairos_temporal_cc(g, int(ta), int(tw), _ptr(out)), "kairos_temporal_cc")
    return out


def kairos_selectivity_build(g, min_degree):
    _check(lib().kairos_selectivity_build(g, int(min_degree)), "kairos_selectivity_build")


def kairos_selectivity_estimate(g, kind, vertices, a, b, tw, want_exact=True):
    """(estimates, exact counts) for the vertices' lists (kind 0 forward, 1 reversed)."""
    v = np.ascontiguousarray(vertices, np.int32)
    est = np.zeros(v.size, np.uint64)
    ex = np.zeros(v.size, np.uint64) if want_exact else None
    _check(lib().kairos_selectivity_estimate(g, int(kind), v.ctypes.data, v.size, int(a), int(b), int(tw),
                                             est.ctypes.data, ex.ctypes.data if want_exact else None),
           "kairos_selectivity_estimate")
    return est, ex


def kairos_selectivity_histogram(g, kind, vertex):
    """(tmin, S, lmin, D), counts[100][100] of one vertex's histogram."""
    meta = np.zeros(4, np.uint64)
    counts = np.zeros(100 * 100, np.uint32)
    _check(lib().kairos_selectivity_histogram(g, int(kind), int(vertex), meta.ctypes.data, counts.ctypes.data),
           "kairos_selectivity_histogram")
    return tuple(int(x) for x in meta), counts.reshape(100, 100)


def kairos_router_create(servers):
    """One submission point over several servers (graph replicas, normally one per GPU)."""
    arr = (_P * len(servers))(*servers)
    r = _P()
    _check(lib().kairos_router_create(arr, len(servers), ctypes.byref(r)), "kairos_router_create")
    return r


def kairos_router_submit(r, query, out) -> int:
    q, _ = make_queries([query])
    t = ctypes.c_uint64(0)
    _check(lib().kairos_router_submit(r, q, _ptr(out), ctypes.byref(t)), "kairos_router_submit")
    return t.value


def kairos_router_poll(r, ticket, timeout_us=-1):
    info = kairos_result_info()
    st = lib().kairos_router_poll(r, int(ticket), int(timeout_us), ctypes.byref(info))
    if st == KAIROS_ERR_NOT_READY:
        return None
    _check(st, "kairos_router_poll")
    return info


def kairos_router_replica_counts(r, n):
    sub = np.zeros(n, np.uint64)
    done = np.zeros(n, np.uint64)
    k = lib().kairos_router_replica_counts(r, sub.ctypes.data, done.ctypes.data, n)
    return sub[:k].tolist(), done[:k].tolist()


def kairos_router_destroy(r):
    lib().kairos_router_destroy(r)


def kairos_last_error() -> str:
    return lib().kairos_last_error().decode()


def kairos_last_kernel_ms(g) -> float:
    return float(lib().kairos_last_kernel_ms(g))


PHASES = ("lane states", "range search", "chunk registration", "local walk", "chunk wait", "chunk walk",
          "grid barrier", "other")


def kairos_last_phase_cycles(g):
    """Per-phase cycles (summed over warps) of the last launch; zeros unless
    KAIROS_PHASE_CLOCK=1 was set before the process started."""
    c = np.zeros(8, np.uint64)
    lib().kairos_last_phase_cycles(g, c.ctypes.data)
    return dict(zip(PHASES, c.tolist()))


STREAM_COUNTERS = ("blocks", "fix_rounds", "fix_vertices", "fix_edges", "candidates", "scanned",
                   "pass_filter_cycles", "fixup_cycles", "barrier_init_readout_cycles", "pass_relax_cycles",
                   "cand_1_lane", "cand_2_4_lanes", "cand_5_16_lanes", "cand_17_64_lanes", "cand_lanes",
                   "cand_improving", "lanes_lowered", "pass_wall_ns", "round_wall_ns", "run_wall_ns",
                   "passes", "grid_rounds", "one_block_runs")


def kairos_last_stream_profile(g):
    """Counters of the last time-ordered (relax_mode 3) launch (cycles and lane counts need
    KAIROS_PHASE_CLOCK=1)."""
    c = np.zeros(len(STREAM_COUNTERS), np.uint64)
    lib().kairos_last_stream_profile(g, c.ctypes.data)
    return dict(zip(STREAM_COUNTERS, c.tolist()))


def kairos_last_round_profile(g, max_rounds=256):
    """(frontier sizes, chunk counts, ms) per round of the last edge-map launch."""
    f = np.zeros(max_rounds, np.uint32)
    c = np.zeros(max_rounds, np.uint32)
    ms = np.zeros(max_rounds, np.float64)
    r = lib().kairos_last_round_profile(g, max_rounds, f.ctypes.data, c.ctypes.data, ms.ctypes.data)
    return f[:r], c[:r], ms[:r]


class Graph:
    """Owning wrapper of a kairos_graph handle."""

    def __init__(self, n_vertices, src, dst, t_dep, lam, stream=None, allocator=None, skip_reverse=False):
        self.n = int(n_vertices)
        self.m = int(src.shape[0])
        self.theta = KAIROS_NO_INDEX
        self.fingerprint = graph_fingerprint(n_vertices, src, dst, t_dep, lam)
        self._allocator = allocator  # keeps the callbacks alive as long as the graph
        self.handle = kairos_graph_build(n_vertices, src, dst, t_dep, lam, stream, allocator, skip_reverse)

    @classmethod
    def from_edges(cls, el, **kw):
        return cls(el.n, el.src, el.dst, el.t, el.lam, **kw)

    def index(self, threshold):
        kairos_index_build(self.handle, threshold)
        self.theta = int(threshold)
        return self

    def earliest_arrival(self, src, ta, tw, out):
        return kairos_earliest_arrival(self.handle, self.n, src, ta, tw, out)

    def latest_departure(self, dst, ta, tw, out):
        return kairos_latest_departure(self.handle, self.n, dst, ta, tw, out)

    def fastest_path(self, src, ta, tw, out, strict=0, want_stats=False):
        return kairos_fastest_path(self.handle, self.n, src, ta, tw, out, strict, want_stats)

    def shortest_duration(self, src, ta, tw, out, strict=0):
        return kairos_shortest_duration(self.handle, self.n, src, ta, tw, out, strict)

    def temporal_bfs(self, src, ta, tw, out, strict=0):
        return kairos_temporal_bfs(self.handle, self.n, src, ta, tw, out, strict)

    def temporal_cc(self, ta, tw, out):
        return kairos_temporal_cc(self.handle, self.n, ta, tw, out)

    def earliest_arrival_noalloc(self, src, ta, tw, out):
        """kairos_earliest_arrival_noalloc: earliest arrival into the device buffer `out`
        (n labels) with no device allocation."""
        return kairos_earliest_arrival_noalloc(self.handle, self.n, src, ta, tw, out)

    def batch(self, queries, out, want_stats=True):
        return kairos_batch_query(self.handle, self.n, queries, out, want_stats)

    def tuning(self):
        return kairos_get_tuning(self.handle)

    def set_tuning(self, **fields):
        return kairos_set_tuning(self.handle, **fields)

    def autotune(self, sample, cache=None, min_lanes=1):
        """Time launch shapes on `sample` (lane widths >= min_lanes) and install the fastest.
        With `cache` (a JSON file path), a shape already found for this graph, index threshold,
        query sample, GPU model and library build is installed without measuring, and a new one
        is stored."""
        if cache is None:
            return kairos_autotune(self.handle, sample, min_lanes)
        key = autotune_cache_key(self, sample) + (f":{min_lanes}" if min_lanes > 1 else "")
        table = _read_cache(cache)
        if key in table:
            return kairos_set_tuning(self.handle, **table[key])
        best = kairos_autotune(self.handle, sample, min_lanes)
        table = _read_cache(cache)  # re-read: another process may have added entries
        table[key] = {name: int(getattr(best, name)) for name, _ in kairos_tuning._fields_}
        _write_cache(cache, table)
        return best

    def autotune_index(self, sample, thetas=(16, 64, 256, 1024, 4096, KAIROS_NO_INDEX)):
        return kairos_autotune_index(self.handle, sample, thetas)

    def info(self):
        return kairos_graph_get_info(self.handle)

    def last_kernel_ms(self):
        return kairos_last_kernel_ms(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            kairos_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
