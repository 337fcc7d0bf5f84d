"""Seeded synthetic temporal graphs and query streams.

The paper's datasets (Table 3) are not available, so seeded R-MAT graphs with skewed
degrees and skewed or bursty departure times stand in for them.  This module draws edge
lists and queries only; it contains none of the temporal-path arithmetic and is the one
module that both the oracle tests and the GPU path use.

Every draw is counter-based (SplitMix64 of seed, item index and draw number), so a
workload is a pure function of its seed and sizes, independent of thread counts, and
identical on x86-64 and AArch64 hosts.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

INF = 0xFFFFFFFF          # "unreached" time label
C_MIRROR = 0xFFFFFFFE     # largest finite time; t + lambda must not exceed it
MASK64 = (1 << 64) - 1

TIME_UNIFORM, TIME_BURSTY, TIME_ZIPF = 0, 1, 2
LAM_UNIFORM, LAM_GEOMETRIC = 0, 1


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64), ("m", ctypes.c_int64), ("scale", ctypes.c_int32),
        ("time_model", ctypes.c_int32), ("a", ctypes.c_double), ("b", ctypes.c_double),
        ("c", ctypes.c_double), ("t_span", ctypes.c_uint64), ("n_bursts", ctypes.c_int32),
        ("burst_frac", ctypes.c_double), ("burst_sigma", ctypes.c_double),
        ("zipf_s", ctypes.c_double), ("lam_model", ctypes.c_int32), ("lam_bits", ctypes.c_int32),
        ("lam_lo", ctypes.c_uint32), ("lam_hi", ctypes.c_uint32), ("lam_mean", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (plain C, gcc, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-fno-semantic-interposition", "-shared", "-pthread",
                                   "-ffp-contract=off",
                                   "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_rmat.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.synth_rmat.restype = ctypes.c_int
        lib.synth_sm64.argtypes = [ctypes.c_uint64]
        lib.synth_sm64.restype = ctypes.c_uint64
        lib.synth_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        lib.synth_draw.restype = ctypes.c_uint64
        for fn in ("synth_det_log", "synth_det_exp"):
            getattr(lib, fn).argtypes = [ctypes.c_double]
            getattr(lib, fn).restype = ctypes.c_double
        lib.synth_zipf_rank.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double]
        lib.synth_zipf_rank.restype = ctypes.c_uint64
        _lib = lib
    return _lib


def lib():
    return _load()


# ---- counter-based draws in Python (same definition as synth.c) ----------------------

def sm64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def draw(seed: int, i: int, d: int) -> int:
    return sm64((seed ^ sm64(((i << 8) | (d & 0xFF)) & MASK64)) & MASK64)


def u01(r: int) -> float:
    return ((r >> 11) + 0.5) * (1.0 / 9007199254740992.0)


def below(r: int, n: int) -> int:
    return ((r >> 32) * n) >> 32


# ---- edge lists ----------------------------------------------------------------------

@dataclass(frozen=True)
class GraphSpec:
    """A seeded R-MAT temporal graph: 2^scale vertices, m edges (u, v, t, lambda)."""
    scale: int
    m: int
    seed: int
    abc: tuple = (0.57, 0.19, 0.19)
    time_model: int = TIME_UNIFORM
    t_span: int = 1 << 20
    n_bursts: int = 10
    burst_frac: float = 0.8
    burst_sigma: float = 4096.0
    zipf_s: float = 1.2
    lam_model: int = LAM_UNIFORM
    lam_lo: int = 1
    lam_hi: int = 100
    lam_mean: float = 50.0
    lam_bits: int = 32

    @property
    def n(self) -> int:
        return 1 << self.scale


@dataclass
class EdgeList:
    """Structure-of-arrays temporal edge list (host memory)."""
    n: int
    src: np.ndarray   # int32[m]
    dst: np.ndarray   # int32[m]
    t: np.ndarray     # uint32[m] departure time
    lam: np.ndarray   # uint32[m] or uint16[m] duration
    spec: GraphSpec | None = None

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def rmat(spec: GraphSpec, nthreads: int = 0) -> EdgeList:
    """Draw the edge list of `spec` (multi-threaded C; thread count does not change it)."""
    L = _load()
    m = int(spec.m)
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    t = np.empty(m, np.uint32)
    lam = np.empty(m, np.uint16 if spec.lam_bits == 16 else np.uint32)
    p = _Params(seed=spec.seed, m=m, scale=spec.scale, time_model=spec.time_model,
                a=spec.abc[0], b=spec.abc[1], c=spec.abc[2], t_span=spec.t_span,
                n_bursts=spec.n_bursts, burst_frac=spec.burst_frac, burst_sigma=spec.burst_sigma,
                zipf_s=spec.zipf_s, lam_model=spec.lam_model, lam_bits=spec.lam_bits,
                lam_lo=spec.lam_lo, lam_hi=spec.lam_hi, lam_mean=spec.lam_mean)
    rc = L.synth_rmat(ctypes.byref(p), src.ctypes.data, dst.ctypes.data, t.ctypes.data,
                      lam.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError(f"synth_rmat rejected {spec}")
    return EdgeList(spec.n, src, dst, t, lam, spec)


def random_small(n: int, m: int, seed: int, t_max: int, lam_max: int, lam_min: int = 0) -> EdgeList:
    """Tiny uniform random multigraph (self-loops and parallel edges allowed) for
    brute-force checks: u, v uniform in [0, n), t in [0, t_max], lambda in [lam_min, lam_max]."""
    src = np.array([below(draw(seed, i, 0), n) for i in range(m)], np.int32)
    dst = np.array([below(draw(seed, i, 1), n) for i in range(m)], np.int32)
    t = np.array([below(draw(seed, i, 2), t_max + 1) for i in range(m)], np.uint32)
    lam = np.array([lam_min + below(draw(seed, i, 3), lam_max - lam_min + 1) for i in range(m)], np.uint32)
    return EdgeList(n, src, dst, t, lam, None)


# ---- queries -------------------------------------------------------------------------

EA, LD = 0, 1


@dataclass(frozen=True)
class Query:
    kind: int      # EA (source = vertex) or LD (target = vertex)
    vertex: int
    ta: int
    tw: int
    strict: int = 0


def degrees(el: EdgeList):
    out_deg = np.bincount(el.src, minlength=el.n)
    in_deg = np.bincount(el.dst, minlength=el.n)
    return out_deg, in_deg


def pick_vertices(el: EdgeList, count: int, seed: int, need_out: bool, need_in: bool) -> list[int]:
    """Uniform vertices, each redrawn (next draw number) until it has the required
    out-degree >= 1 and/or in-degree >= 1."""
    out_deg, in_deg = degrees(el)
    ok = np.ones(el.n, bool)
    if need_out:
        ok &= out_deg > 0
    if need_in:
        ok &= in_deg > 0
    if not ok.any():
        raise ValueError("no vertex satisfies the degree requirement")
    res = []
    for q in range(count):
        d = 0
        while True:
            v = below(draw(seed, q, d % 256), el.n) if d < 256 else below(draw(seed ^ d, q, 0), el.n)
            if ok[v]:
                break
            d += 1
        res.append(int(v))
    return res


def random_windows(count: int, seed: int, span: int, lo_frac: float, hi_frac: float):
    """Window length L = floor(span * U(lo_frac, hi_frac)), ta ~ U[0, span - L], tw = ta + L - 1."""
    res = []
    for q in range(count):
        f = lo_frac + (hi_frac - lo_frac) * u01(draw(seed, q, 200))
        L = max(1, int(math.floor(span * f)))
        ta = below(draw(seed, q, 201), span - L + 1)
        res.append((ta, ta + L - 1))
    return res


def log_uniform_windows(count: int, seed: int, span: int, lo_log2: float, hi_log2: float):
    """Window length L = floor(2^U(lo_log2, hi_log2)) (capped at span), placed uniformly."""
    res = []
    for q in range(count):
        e = lo_log2 + (hi_log2 - lo_log2) * u01(draw(seed, q, 210))
        L = min(span, max(1, int(math.floor(2.0 ** e))))
        ta = below(draw(seed, q, 211), span - L + 1)
        res.append((ta, ta + L - 1))
    return res


# ---- the five workloads ---------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    key: int
    name: str
    graph: GraphSpec
    description: str
    theta: int = 0xFFFFFFFF    # selective-index degree threshold (UINT32_MAX: none)


_G = 0x4B410000

WORKLOADS = {
    1: Workload(1, "tiny", GraphSpec(scale=13, m=100_000, seed=_G + 1, time_model=TIME_UNIFORM,
                                     t_span=1 << 20, lam_model=LAM_UNIFORM, lam_lo=1, lam_hi=100),
                "R-MAT 2^13 vertices, 1e5 edges, t~U[0,2^20), lambda~U[1,100]; one EA query, "
                "window [0, 2^20-1]"),
    2: Workload(2, "medium", GraphSpec(scale=20, m=1 << 25, seed=_G + 2, time_model=TIME_BURSTY,
                                       t_span=1 << 24, n_bursts=10, burst_frac=0.8,
                                       burst_sigma=4096.0, lam_model=LAM_GEOMETRIC, lam_mean=50.0),
                "R-MAT scale 20, edge factor 32; t: 80% in 10 Gaussian bursts (sigma 2^12), 20% "
                "U[0,2^24); lambda geometric mean 50; 64 sources x (EA + LD), full window",
                theta=256),
    3: Workload(3, "batched", GraphSpec(scale=24, m=1 << 28, seed=_G + 3, time_model=TIME_UNIFORM,
                                        t_span=1 << 28, lam_model=LAM_UNIFORM, lam_lo=1, lam_hi=1000),
                "R-MAT scale 24, edge factor 16; t~U[0,2^28), lambda~U[1,1000]; 256 EA queries, "
                "random sources, window length U(1%,100%) of the span"),
    4: Workload(4, "served", GraphSpec(scale=24, m=1 << 28, seed=_G + 3, time_model=TIME_UNIFORM,
                                       t_span=1 << 28, lam_model=LAM_UNIFORM, lam_lo=1, lam_hi=1000),
                "workload 3's graph resident; Poisson stream, 70% EA / 30% LD, window length "
                "log-uniform 2^10..2^28"),
    5: Workload(5, "large-skewed", GraphSpec(scale=26, m=1 << 31, seed=_G + 5, abc=(0.65, 0.15, 0.15),
                                             time_model=TIME_ZIPF, t_span=1 << 31, zipf_s=1.2,
                                             lam_model=LAM_UNIFORM, lam_lo=1, lam_hi=4096, lam_bits=16),
                "R-MAT scale 26 (a=.65), edge factor 32; t Zipf(1.2) over [0,2^31); lambda~U[1,4096] "
                "uint16; 64 EA/LD, full window"),
}


def scaled(spec: GraphSpec, scale: int, m: int) -> GraphSpec:
    """Same laws and seed at a smaller size (time span kept)."""
    return replace(spec, scale=scale, m=m)


def workload_queries(key: int, el: EdgeList, count: int | None = None, shard: int = 0) -> list[Query]:
    """The query set of workload `key` drawn on edge list `el` (seed = graph seed + 0x100);
    shard > 0 draws a disjointly seeded set of the same shape (one per replica)."""
    w = WORKLOADS[key]
    seed = w.graph.seed + 0x100 + key + 0x10000 * shard
    span = w.graph.t_span
    if key == 1:
        (s,) = pick_vertices(el, 1, seed, True, False)
        return [Query(EA, s, 0, (1 << 20) - 1)]
    if key in (2, 5):
        k = 64 if count is None else count
        vs = pick_vertices(el, k, seed, True, True)
        return [Query(EA, v, 0, C_MIRROR) for v in vs] + [Query(LD, v, 0, C_MIRROR) for v in vs]
    if key == 3:
        k = 256 if count is None else count
        vs = pick_vertices(el, k, seed, True, False)
        wins = random_windows(k, seed, span, 0.01, 1.0)
        return [Query(EA, v, ta, tw) for v, (ta, tw) in zip(vs, wins)]
    if key == 4:
        k = 1024 if count is None else count
        kinds = [EA if u01(draw(seed, q, 220)) < 0.7 else LD for q in range(k)]
        v_ea = pick_vertices(el, k, seed, True, False)
        v_ld = pick_vertices(el, k, seed ^ 0x1D, False, True)
        wins = log_uniform_windows(k, seed, span, 10.0, 28.0)
        return [Query(kd, (v_ea[q] if kd == EA else v_ld[q]), ta, tw)
                for q, (kd, (ta, tw)) in enumerate(zip(kinds, wins))]
    raise KeyError(key)


def poisson_arrivals(count: int, rate_hz: float, seed: int) -> np.ndarray:
    """Open-loop arrival offsets (seconds) of a Poisson stream, drawn before the run."""
    gaps = np.array([-math.log(u01(draw(seed, q, 230))) / rate_hz for q in range(count)])
    return np.cumsum(gaps)
