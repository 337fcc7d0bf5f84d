"""ORACLE -- test infrastructure only.

Plain statement of the selective-access pieces of Sec. 5 (cost model, Eqs. 1-3; cardinality
estimation, Sec. 5.2): the per-vertex 2D density histogram over (start time, duration), the
estimate of how many of a vertex's edges satisfy a temporal predicate, the exact count, the
access decision of Eq. 3, and the estimator-accuracy measure of Sec. 6.5.  Only the test suite
and the benchmark use it; it shares no code with the CUDA library.  All arithmetic is exact
integer arithmetic (Python ints), so the GPU's results must match bit for bit.

Readings (the paper fixes the bucket count, 100 per dimension, and "equally divided" ranges,
but not the range, the bucket rule or how a bucket counts towards a predicate):
  * a vertex's histogram spans its own edges: starts [tmin, tmax], durations [lmin, lmax];
    with S = tmax - tmin + 1 and D = lmax - lmin + 1, an edge (t, lam) falls in bucket
    i = floor((t - tmin) * 100 / S), j = floor((lam - lmin) * 100 / D);
  * bucket i holds the integer starts [tmin + ceil(i S / 100), tmin + ceil((i + 1) S / 100) - 1]
    (possibly none), and its centre is the floor of the mean of those two ends (likewise j);
  * the estimate of a predicate counts every edge of a bucket whose centre satisfies it: for
    the edge-map's predicate (departure in [a, b], arrival t + lam <= tw) that is the sum of
    c[i][j] over buckets with a <= centre_i <= b and centre_i + centre_j <= tw;
  * Eq. 3 with selectivity beta = k / deg(v): the index is used when beta <= theta_sel,
    i.e. 1000 * k <= theta_permille * deg (theta_sel in parts per thousand);
  * accuracy (Sec. 6.5): over the vertices with degree >= the cutoff and a window [T_X, max]
    whose start T_X is the departure time above which X percent of all edges depart, the
    fraction of vertices where the decision from the estimate equals the decision from the
    exact count, at theta_sel = 20%.
"""
from __future__ import annotations

import numpy as np

BUCKETS = 100


def _cdiv(a: int, b: int) -> int:
    return -((-a) // b)


def bucket_ends(lo: int, span: int, i: int):
    """First and last integer of bucket i of [lo, lo + span); (x, x - 1) when it holds none."""
    return lo + _cdiv(i * span, BUCKETS), lo + _cdiv((i + 1) * span, BUCKETS) - 1


def bucket_centre(lo: int, span: int, i: int) -> int:
    a, b = bucket_ends(lo, span, i)
    return (a + b) // 2


class VertexHistogram:
    """The 100 x 100 (start, duration) density histogram of one vertex's edges."""

    def __init__(self, t, lam):
        t = [int(x) for x in t]
        lam = [int(x) for x in lam]
        if not t:
            raise ValueError("a histogram needs at least one edge")
        self.tmin, self.lmin = min(t), min(lam)
        self.S = max(t) - self.tmin + 1
        self.D = max(lam) - self.lmin + 1
        self.deg = len(t)
        self.counts = [[0] * BUCKETS for _ in range(BUCKETS)]
        for x, y in zip(t, lam):
            i = (x - self.tmin) * BUCKETS // self.S
            j = (y - self.lmin) * BUCKETS // self.D
            self.counts[i][j] += 1

    def estimate(self, a: int, b: int, tw: int) -> int:
        """Edges counted towards departure in [a, b] and arrival <= tw (bucket centres)."""
        k = 0
        for i in range(BUCKETS):
            s0, s1 = bucket_ends(self.tmin, self.S, i)
            if s0 > s1:
                continue
            sc = (s0 + s1) // 2
            if not (a <= sc <= b):
                continue
            for j in range(BUCKETS):
                if self.counts[i][j] and sc + bucket_centre(self.lmin, self.D, j) <= tw:
                    k += self.counts[i][j]
        return k

    def meta(self):
        return self.tmin, self.S, self.lmin, self.D


def exact_count(t, lam, a: int, b: int, tw: int) -> int:
    """Edges of a vertex with departure in [a, b] and arrival t + lam <= tw."""
    t = np.asarray(t, np.int64)
    lam = np.asarray(lam, np.int64)
    return int(((t >= a) & (t <= b) & (t + lam <= tw)).sum())


def use_index(k: int, deg: int, theta_permille: int) -> bool:
    """Eq. 3: the index (T_v) when the selectivity k / deg is at most theta_sel."""
    return 1000 * k <= theta_permille * deg


def recent_start(t_all, percent: float) -> int:
    """T_X: the departure time at or above which `percent` of all edges depart (the smallest
    time with at most that share of edges strictly after it... read as the (100 - X)th
    percentile of departures, taken as an order statistic)."""
    s = np.sort(np.asarray(t_all, np.int64))
    k = int(np.floor(len(s) * (1.0 - percent / 100.0)))
    k = min(max(k, 0), len(s) - 1)
    return int(s[k])


def accuracy(el, cutoff: int, percent: float, theta_permille: int = 200, tw: int = 0xFFFFFFFE):
    """Sec. 6.5 estimator accuracy on the out-lists of el: (vertices judged, agreements)."""
    src = np.asarray(el.src, np.int64)
    order = np.argsort(src, kind="stable")
    deg = np.bincount(src, minlength=el.n)
    off = np.concatenate([[0], np.cumsum(deg)])
    T = recent_start(el.t, percent)
    judged = agree = 0
    for u in np.flatnonzero(deg >= cutoff):
        e = order[off[u]:off[u + 1]]
        t, lam = el.t[e], el.lam[e]
        h = VertexHistogram(t, lam)
        est = h.estimate(T, tw, tw)
        ex = exact_count(t, lam, T, tw, tw)
        judged += 1
        agree += use_index(est, h.deg, theta_permille) == use_index(ex, h.deg, theta_permille)
    return judged, agree
