"""ORACLE -- test infrastructure only.

Plain CPU statement of the temporal path queries (earliest arrival, latest departure,
fastest path, shortest duration, temporal BFS) and of temporal connected components,
used by the test suite, the package smoke check and the CPU-baseline leg of the
benchmark, and by nothing in the library.  `oracle.c` holds the single-threaded one-pass
scans; this module loads it and adds pure-Python brute force over simple paths for tiny
graphs.  It shares no code with the CUDA library and imports only numpy and ctypes; edge
lists are passed in as any object with n, src, dst, t and lam attributes.

Semantics (the paper's Sec. 2.1 edge model, Sec. 2.2 ordering predicates, Alg. 2 as read
with the source initialised to the window start):
  * edge (u, v, t, lam) departs u at t, arrives at v at t + lam;
  * window [ta, tw] inclusive: usable edges have t >= ta and t + lam <= tw;
  * consecutive edges e, f of a path: t_f >= t_e + lam_e (Succeeds) or > (StrictlySucceeds);
    the first edge may depart at ta and the last may arrive at tw under either predicate;
  * EA[s] = ta; EA[v] = min arrival over paths s -> v; LD[x] = tw; LD[u] = max first
    departure over paths u -> x; FP[s] = 0; FP[v] = min (arrival - first departure) over
    paths s -> v; SD[s] = 0; SD[v] = min sum of durations over paths s -> v; temporal BFS:
    the least number of edges of a path s -> v; unreachable = 0xFFFFFFFF.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

UNREACHED = 0xFFFFFFFF
C_MIRROR = 0xFFFFFFFE
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, plain C)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_time_order.argtypes = [ctypes.c_int64, _P, _P]
        L.oracle_time_order.restype = ctypes.c_int
        for fn in ("oracle_earliest_arrival", "oracle_latest_departure", "oracle_fastest",
                   "oracle_shortest_duration", "oracle_temporal_bfs"):
            f = getattr(L, fn)
            f.argtypes = [ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, _P, ctypes.c_int32,
                          ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, _P]
            f.restype = ctypes.c_int
        L.oracle_admissible_ea.argtypes = [ctypes.c_int64, _P, _P, _P, _P, ctypes.c_int32,
                                           ctypes.c_uint32, ctypes.c_int]
        L.oracle_admissible_ea.restype = ctypes.c_uint64
        L.oracle_admissible_ld.argtypes = [ctypes.c_int64, _P, _P, _P, _P, ctypes.c_int32,
                                           ctypes.c_uint32, ctypes.c_int]
        L.oracle_admissible_ld.restype = ctypes.c_uint64
        L.oracle_certify_ea.argtypes = [ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, ctypes.c_int32,
                                        ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, _P,
                                        ctypes.POINTER(ctypes.c_int64)]
        L.oracle_certify_ea.restype = ctypes.c_int
        L.oracle_certify_ea_rows.argtypes = [ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, ctypes.c_int,
                                             _P, _P, _P, _P, _P, _P, _P]
        L.oracle_certify_ea_rows.restype = ctypes.c_int
        L.oracle_temporal_cc.argtypes = [ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, ctypes.c_uint32,
                                         ctypes.c_uint32, _P]
        L.oracle_temporal_cc.restype = ctypes.c_int
        _lib = L
    return _lib


def _arrays(el):
    src = np.ascontiguousarray(el.src, np.int32)
    dst = np.ascontiguousarray(el.dst, np.int32)
    t = np.ascontiguousarray(el.t, np.uint32)
    lam = np.ascontiguousarray(el.lam, np.uint32)  # widened copy when durations are uint16
    return src, dst, t, lam


class Oracle:
    """The oracle bound to one edge list: sorts it by departure time once (stable radix sort), then
    answers queries by the one-pass scans of oracle.c."""

    def __init__(self, el):
        self.n = int(el.n)
        self.src, self.dst, self.t, self.lam = _arrays(el)
        self.m = int(self.src.shape[0])
        self.perm = np.empty(self.m, np.uint32)
        L = _load()
        if L.oracle_time_order(self.m, self.t.ctypes.data, self.perm.ctypes.data) != 0:
            raise MemoryError("oracle_time_order failed")

    def _ptrs(self):
        return (self.src.ctypes.data, self.dst.ctypes.data, self.t.ctypes.data,
                self.lam.ctypes.data, self.perm.ctypes.data)

    def earliest_arrival(self, s: int, ta: int, tw: int, strict: int = 0) -> np.ndarray:
        out = np.empty(self.n, np.uint32)
        rc = _load().oracle_earliest_arrival(self.n, self.m, *self._ptrs(), int(s), int(ta), int(tw),
                                             int(strict), out.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_earliest_arrival: invalid arguments")
        return out

    def latest_departure(self, x: int, ta: int, tw: int, strict: int = 0) -> np.ndarray:
        out = np.empty(self.n, np.uint32)
        rc = _load().oracle_latest_departure(self.n, self.m, *self._ptrs(), int(x), int(ta), int(tw),
                                             int(strict), out.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_latest_departure: invalid arguments")
        return out

    def fastest(self, s: int, ta: int, tw: int, strict: int = 0) -> np.ndarray:
        """Fastest-path durations from s (min arrival - first departure; fp[s] = 0)."""
        out = np.empty(self.n, np.uint32)
        rc = _load().oracle_fastest(self.n, self.m, *self._ptrs(), int(s), int(ta), int(tw), int(strict),
                                    out.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_fastest: invalid arguments or allocation failure")
        return out

    def shortest_duration(self, s: int, ta: int, tw: int, strict: int = 0) -> np.ndarray:
        """Shortest-duration labels from s (least total travel time; sd[s] = 0)."""
        out = np.empty(self.n, np.uint32)
        rc = _load().oracle_shortest_duration(self.n, self.m, *self._ptrs(), int(s), int(ta), int(tw),
                                              int(strict), out.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_shortest_duration: invalid arguments or allocation failure")
        return out

    def temporal_bfs(self, s: int, ta: int, tw: int, strict: int = 0) -> np.ndarray:
        """Temporal BFS levels from s (least number of edges of a time-respecting path)."""
        out = np.empty(self.n, np.uint32)
        rc = _load().oracle_temporal_bfs(self.n, self.m, *self._ptrs(), int(s), int(ta), int(tw), int(strict),
                                         out.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_temporal_bfs: invalid arguments or allocation failure")
        return out

    def query(self, q) -> np.ndarray:
        """q has .kind (0 EA, 1 LD), .vertex, .ta, .tw, .strict."""
        if q.kind == 0:
            return self.earliest_arrival(q.vertex, q.ta, q.tw, q.strict)
        return self.latest_departure(q.vertex, q.ta, q.tw, q.strict)

    def admissible(self, q, labels: np.ndarray) -> int:
        """TE(q): edges usable under the final labels of query q."""
        labels = np.ascontiguousarray(labels, np.uint32)
        L = _load()
        if q.kind == 0:
            return int(L.oracle_admissible_ea(self.m, self.src.ctypes.data, self.t.ctypes.data,
                                              self.lam.ctypes.data, labels.ctypes.data, int(q.vertex),
                                              int(q.tw), int(q.strict)))
        return int(L.oracle_admissible_ld(self.m, self.dst.ctypes.data, self.t.ctypes.data,
                                          self.lam.ctypes.data, labels.ctypes.data, int(q.vertex),
                                          int(q.ta), int(q.strict)))


def temporal_cc(el, ta: int, tw: int) -> np.ndarray:
    """Temporal connected components in [ta, tw] (see oracle.c): the smallest vertex id of each
    vertex's component in the undirected graph of the window's usable edges."""
    src, dst, t, lam = _arrays(el)
    out = np.empty(int(el.n), np.uint32)
    rc = _load().oracle_temporal_cc(int(el.n), int(src.shape[0]), src.ctypes.data, dst.ctypes.data, t.ctypes.data,
                                    lam.ctypes.data, int(ta), int(tw), out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_temporal_cc: invalid arguments or allocation failure")
    return out


def brute_temporal_cc(n, src, dst, t, lam, ta, tw):
    """Components by breadth-first search over the window's usable edges (tiny graphs)."""
    adj = [[] for _ in range(n)]
    for u, v, x, y in zip(src, dst, t, lam):
        if _usable(int(x), int(y), ta, tw):
            adj[int(u)].append(int(v))
            adj[int(v)].append(int(u))
    out = [None] * n
    for s in range(n):
        if out[s] is not None:
            continue
        comp, stack = [s], [s]
        out[s] = -1
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if out[y] is None:
                    out[y] = -1
                    comp.append(y)
                    stack.append(y)
        for x in comp:
            out[x] = min(comp)
    return np.array(out, np.uint32)


def certify_ea(el, s: int, ta: int, tw: int, strict: int, labels: np.ndarray):
    """Certificate check of earliest-arrival labels at any size (see oracle.c).
    Returns (status, bad): 0 holds, 1 fails at `bad`, 2 not applicable (lam == 0, Succeeds)."""
    src, dst, t, lam = _arrays(el)
    labels = np.ascontiguousarray(labels, np.uint32)
    bad = ctypes.c_int64(0)
    rc = _load().oracle_certify_ea(int(el.n), int(src.shape[0]), src.ctypes.data, dst.ctypes.data,
                                   t.ctypes.data, lam.ctypes.data, int(s), int(ta), int(tw), int(strict),
                                   labels.ctypes.data, ctypes.byref(bad))
    if rc < 0:
        raise ValueError("oracle_certify_ea: invalid arguments")
    return rc, int(bad.value)


def mirror_edges(src, dst, t, lam):
    """Reverse, time-mirrored edge list: (v, u, C - (t + lam), lam).  A path u -> x that
    departs at t1 maps to a path x -> u arriving at C - t1, so latest departure in [ta, tw]
    equals C minus earliest arrival on the mirror in [C - tw, C - ta]."""
    t2 = (np.uint64(C_MIRROR) - (t.astype(np.uint64) + lam.astype(np.uint64))).astype(np.uint32)
    return dst.copy(), src.copy(), t2, lam.astype(np.uint32)


class Certifier:
    """The any-size certificate (`certify_ea` above) for many queries of both kinds on one
    edge list, with the arrays converted once.  Latest-departure labels are certified
    through the mirror identity of `mirror_edges`: LD[u] = C - EA'[u], where EA' is
    earliest arrival from the target on the reversed graph with departures C - (t + lam)
    over the window [C - tw, C - ta] (same predicate).  The mirrored graph reuses the
    source and head arrays (swapped) and adds only its departure times, computed in chunks.
    `check_all` runs the single-threaded C checks of independent queries on a thread pool
    (the C calls release the interpreter lock)."""

    def __init__(self, el):
        self.n = int(el.n)
        self.src, self.dst, self.t, self.lam = _arrays(el)
        self.m = int(self.src.shape[0])
        self._t_mirror = None
        self._mu = threading.Lock()

    def _mirror_times(self):
        with self._mu:
            if self._t_mirror is None:
                t2 = np.empty(self.m, np.uint32)
                step = 1 << 24
                for a in range(0, self.m, step):
                    b = min(self.m, a + step)
                    t2[a:b] = (np.uint64(C_MIRROR) - (self.t[a:b].astype(np.uint64) +
                                                      self.lam[a:b].astype(np.uint64))).astype(np.uint32)
                self._t_mirror = t2
        return self._t_mirror

    def check(self, q, labels):
        """(status, bad) of one query's labels: 0 holds, 1 fails, 2 not applicable."""
        labels = np.ascontiguousarray(labels, np.uint32)
        bad = ctypes.c_int64(0)
        if q.kind == 0:
            src, dst, t, ta, tw, lab = self.src, self.dst, self.t, q.ta, q.tw, labels
        else:
            src, dst, t = self.dst, self.src, self._mirror_times()
            ta, tw = C_MIRROR - q.tw, C_MIRROR - q.ta
            lab = np.where(labels == UNREACHED, np.uint32(UNREACHED),
                           (np.uint32(C_MIRROR) - labels).astype(np.uint32))
        rc = _load().oracle_certify_ea(self.n, self.m, src.ctypes.data, dst.ctypes.data, t.ctypes.data,
                                       self.lam.ctypes.data, int(q.vertex), int(ta), int(tw), int(q.strict),
                                       lab.ctypes.data, ctypes.byref(bad))
        if rc < 0:
            raise ValueError("oracle_certify_ea: invalid arguments")
        return rc, int(bad.value)

    def check_group(self, queries, labels):
        """Certify up to 32 queries of one kind in one pass over the edges (the rows form of
        the certificate); labels[i] (a sequence, or a callable of i) is query i's label
        array, fetched one at a time.  Returns [(status, bad)]."""
        w = len(queries)
        assert 1 <= w <= 32 and len({q.kind for q in queries}) == 1
        ld = queries[0].kind == 1
        rows = np.empty((self.n, w), np.uint32)  # vertex-major: the w labels of a vertex together
        for i in range(w):
            lab = np.asarray(labels(i) if callable(labels) else labels[i], np.uint32)
            rows[:, i] = (np.where(lab == UNREACHED, np.uint32(UNREACHED),
                                   (np.uint32(C_MIRROR) - lab).astype(np.uint32)) if ld else lab)
        s = np.array([q.vertex for q in queries], np.int32)
        ta = np.array([C_MIRROR - q.tw if ld else q.ta for q in queries], np.uint32)
        tw = np.array([C_MIRROR - q.ta if ld else q.tw for q in queries], np.uint32)
        st = np.array([q.strict for q in queries], np.int32)
        status = np.zeros(w, np.int32)
        bad = np.zeros(w, np.int64)
        src, dst, t = (self.dst, self.src, self._mirror_times()) if ld else (self.src, self.dst, self.t)
        rc = _load().oracle_certify_ea_rows(self.n, self.m, src.ctypes.data, dst.ctypes.data, t.ctypes.data,
                                            self.lam.ctypes.data, w, s.ctypes.data, ta.ctypes.data,
                                            tw.ctypes.data, st.ctypes.data, rows.ctypes.data,
                                            status.ctypes.data, bad.ctypes.data)
        if rc < 0:
            raise ValueError("oracle_certify_ea_rows: invalid arguments")
        return [(int(a), int(b)) for a, b in zip(status, bad)]

    def check_all(self, queries, rows, threads=None, group=None):
        """Certify query i against rows(i) (a callable returning that query's labels as a
        host array) for every i: queries of one kind are certified `group` at a time in one
        edge pass (default: enough groups to occupy `threads`, at most 16 queries each),
        `threads` groups at once.  Returns the list of (status, bad) in order."""
        from concurrent.futures import ThreadPoolExecutor
        if any(q.kind == 1 for q in queries):
            self._mirror_times()
        cores = threads or os.cpu_count() or 1
        if group is None:
            group = max(1, min(16, -(-len(queries) // cores)))
        groups = []
        for kind in (0, 1):
            idx = [i for i, q in enumerate(queries) if q.kind == kind]
            groups += [idx[c:c + group] for c in range(0, len(idx), group)]
        threads = min(len(groups), cores) or 1
        out = [None] * len(queries)

        def run(gi):
            for i, r in zip(gi, self.check_group([queries[i] for i in gi], lambda k: rows(gi[k]))):
                out[i] = r

        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(run, groups))
        return out


# ---- brute force over simple paths (pure Python, tiny graphs only) ---------------------

def _usable(t, lam, ta, tw):
    return t >= ta and t + lam <= tw


def brute_earliest_arrival(n, src, dst, t, lam, s, ta, tw, strict=0, used=None):
    """Enumerate every vertex-simple time-respecting path from s (a cycle can always be cut
    out of a time-respecting walk without delaying its end) and keep the minimum arrival.
    If `used` is a set, it receives every edge that can extend some such path."""
    out = [UNREACHED] * n
    out[s] = ta
    adj = [[] for _ in range(n)]
    for e in range(len(src)):
        adj[int(src[e])].append(e)

    def go(u, arrival, first, onpath):
        for e in adj[u]:
            te, le = int(t[e]), int(lam[e])
            if not _usable(te, le, ta, tw):
                continue
            if not first and (te <= arrival if strict else te < arrival):
                continue
            if used is not None:
                used.add(e)
            v = int(dst[e])
            if v in onpath:
                continue
            if te + le < out[v]:
                out[v] = te + le
            onpath.add(v)
            go(v, te + le, False, onpath)
            onpath.discard(v)

    go(s, ta, True, {s})
    return np.array(out, np.uint32)


def brute_latest_departure(n, src, dst, t, lam, x, ta, tw, strict=0, used=None):
    """Enumerate every vertex-simple time-respecting path into x, walking backwards, and
    keep the maximum first departure per start vertex.  If `used` is a set, it receives
    every edge that can precede some such path."""
    out = [UNREACHED] * n
    out[x] = tw
    radj = [[] for _ in range(n)]
    for e in range(len(src)):
        radj[int(dst[e])].append(e)

    def go(v, bound, last, onpath):
        # bound: departure time of the path's next edge out of v (tw when v is the target)
        for e in radj[v]:
            te, le = int(t[e]), int(lam[e])
            if not _usable(te, le, ta, tw):
                continue
            if not last and (te + le >= bound if strict else te + le > bound):
                continue
            if used is not None:
                used.add(e)
            u = int(src[e])
            if u in onpath:
                continue
            if out[u] == UNREACHED or te > out[u]:
                out[u] = te
            onpath.add(u)
            go(u, te, False, onpath)
            onpath.discard(u)

    go(x, tw, True, {x})
    return np.array(out, np.uint32)


def brute_fastest(n, src, dst, t, lam, s, ta, tw, strict=0):
    """Enumerate every vertex-simple time-respecting path from s and keep, per end vertex,
    the minimum of (arrival - first departure).  Cutting a cycle out of a time-respecting
    walk keeps its end and moves its first departure no earlier, so simple paths suffice."""
    out = [UNREACHED] * n
    out[s] = 0
    adj = [[] for _ in range(n)]
    for e in range(len(src)):
        adj[int(src[e])].append(e)

    def go(u, arrival, start, onpath):
        for e in adj[u]:
            te, le = int(t[e]), int(lam[e])
            if not _usable(te, le, ta, tw):
                continue
            first = start is None
            if not first and (te <= arrival if strict else te < arrival):
                continue
            v = int(dst[e])
            if v in onpath:
                continue
            st = te if first else start
            if te + le - st < out[v]:
                out[v] = te + le - st
            onpath.add(v)
            go(v, te + le, st, onpath)
            onpath.discard(v)

    go(s, ta, None, {s})
    return np.array(out, np.uint32)


def brute_shortest_duration(n, src, dst, t, lam, s, ta, tw, strict=0):
    """Enumerate every vertex-simple time-respecting path from s and keep, per end vertex,
    the minimum total duration.  Cutting a cycle out of a time-respecting walk keeps it
    time-respecting and removes non-negative durations, so simple paths suffice."""
    out = [UNREACHED] * n
    out[s] = 0
    adj = [[] for _ in range(n)]
    for e in range(len(src)):
        adj[int(src[e])].append(e)

    def go(u, arrival, total, first, onpath):
        for e in adj[u]:
            te, le = int(t[e]), int(lam[e])
            if not _usable(te, le, ta, tw):
                continue
            if not first and (te <= arrival if strict else te < arrival):
                continue
            v = int(dst[e])
            if v in onpath:
                continue
            if total + le < out[v]:
                out[v] = total + le
            onpath.add(v)
            go(v, te + le, total + le, False, onpath)
            onpath.discard(v)

    go(s, ta, 0, True, {s})
    return np.array(out, np.uint32)


def brute_temporal_bfs(n, src, dst, t, lam, s, ta, tw, strict=0):
    """Least number of edges over vertex-simple time-respecting paths from s (a cycle cut out of
    a time-respecting walk leaves a shorter time-respecting walk)."""
    out = [UNREACHED] * n
    out[s] = 0
    adj = [[] for _ in range(n)]
    for e in range(len(src)):
        adj[int(src[e])].append(e)

    def go(u, arrival, hops, first, onpath):
        for e in adj[u]:
            te, le = int(t[e]), int(lam[e])
            if not _usable(te, le, ta, tw):
                continue
            if not first and (te <= arrival if strict else te < arrival):
                continue
            v = int(dst[e])
            if v in onpath:
                continue
            if hops + 1 < out[v]:
                out[v] = hops + 1
            onpath.add(v)
            go(v, te + le, hops + 1, False, onpath)
            onpath.discard(v)

    go(s, ta, 0, True, {s})
    return np.array(out, np.uint32)
