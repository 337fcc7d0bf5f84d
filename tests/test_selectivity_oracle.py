"""Pins for the selective-access oracle (Sec. 5.1 cost model, Sec. 5.2 histogram estimator,
Sec. 6.5 accuracy measure), checked against things other than its own formulas: the bucket
ranges partition the vertex's span and each edge lies in its bucket's range; the estimate is
exact when every edge sits at a bucket centre, equals the degree for a predicate that admits
everything and zero for one that admits nothing, and grows with the predicate; the access
decision follows Eq. 3 at its boundary; and the recent-window start leaves the stated share
of edges.  CPU only."""
import numpy as np
import pytest

import synth
from oracle import selectivity as sel


def random_vertex(rng, deg, t_span, lam_hi):
    t = rng.integers(0, t_span, deg)
    lam = rng.integers(1, lam_hi + 1, deg)
    return t, lam


@pytest.mark.parametrize("span", [1, 7, 99, 100, 101, 12345, 1 << 31])
def test_buckets_partition_the_span(span):
    ends = [sel.bucket_ends(1000, span, i) for i in range(sel.BUCKETS)]
    assert ends[0][0] == 1000 and ends[-1][1] == 1000 + span - 1
    for (a0, b0), (a1, b1) in zip(ends, ends[1:]):
        assert a1 == b0 + 1  # contiguous, possibly empty buckets when span < 100
    assert sum(b - a + 1 for a, b in ends) == span


def test_every_edge_lies_in_its_bucket_range():
    rng = np.random.default_rng(0x5E1)
    for deg, span, lam_hi in ((1, 10, 1), (50, 37, 5), (3000, 1 << 28, 1000), (500, 150, 4096)):
        t, lam = random_vertex(rng, deg, span, lam_hi)
        h = sel.VertexHistogram(t, lam)
        assert sum(map(sum, h.counts)) == deg
        for x, y in zip(t.tolist(), lam.tolist()):
            i = (x - h.tmin) * 100 // h.S
            j = (y - h.lmin) * 100 // h.D
            a, b = sel.bucket_ends(h.tmin, h.S, i)
            c, d = sel.bucket_ends(h.lmin, h.D, j)
            assert a <= x <= b and c <= y <= d


def test_estimate_is_exact_for_unit_buckets():
    """Starts spanning exactly 100 instants and durations exactly 100 values: every bucket
    holds one integer, every edge sits at its bucket's centre, and the estimate is the exact
    count for any predicate."""
    rng = np.random.default_rng(0x5E2)
    t = np.concatenate([[700, 799], rng.integers(700, 800, 3000)])
    lam = np.concatenate([[5, 104], rng.integers(5, 105, 3000)])
    h = sel.VertexHistogram(t, lam)
    assert h.meta() == (700, 100, 5, 100)
    for _ in range(400):
        a, b = sorted(rng.integers(690, 810, 2).tolist())
        tw = int(rng.integers(690, 920))
        assert h.estimate(a, b, tw) == sel.exact_count(t, lam, a, b, tw)


def test_estimate_equals_the_centre_rule_edge_by_edge():
    """For wide buckets the estimate counts each edge by its bucket's centre: recomputed edge
    by edge, finding the bucket by scanning the bucket ranges."""
    rng = np.random.default_rng(0x5E4)
    t, lam = random_vertex(rng, 2500, 1 << 26, 4096)
    h = sel.VertexHistogram(t, lam)
    sr = [sel.bucket_ends(h.tmin, h.S, i) for i in range(100)]
    lr = [sel.bucket_ends(h.lmin, h.D, j) for j in range(100)]
    centre = lambda rs, x: next((a + b) // 2 for a, b in rs if a <= x <= b)
    sc = np.array([centre(sr, x) for x in t.tolist()], np.int64)
    dc = np.array([centre(lr, y) for y in lam.tolist()], np.int64)
    for _ in range(200):
        a, b = sorted(rng.integers(int(t.min()) - 5, int(t.max()) + 5, 2).tolist())
        tw = int(rng.integers(int(t.min()), int(t.max()) + 5000))
        assert h.estimate(a, b, tw) == int(((sc >= a) & (sc <= b) & (sc + dc <= tw)).sum())


def test_estimate_bounds_and_monotonicity():
    rng = np.random.default_rng(0x5E3)
    t, lam = random_vertex(rng, 5000, 1 << 24, 300)
    h = sel.VertexHistogram(t, lam)
    big = 0xFFFFFFFE
    assert h.estimate(0, big, big) == 5000
    assert h.estimate(10, 9, big) == 0
    assert h.estimate(0, big, int(t.min()) - 1) == 0
    prev = -1
    for b in np.linspace(int(t.min()), int(t.max()), 40).astype(int).tolist():
        e = h.estimate(int(t.min()), b, big)
        assert e >= prev
        prev = e
    prev = -1
    for tw in np.linspace(int(t.min()), int(t.max()) + 300, 40).astype(int).tolist():
        e = h.estimate(0, big, tw)
        assert e >= prev
        prev = e


def test_access_decision_follows_eq3():
    assert sel.use_index(200, 1000, 200)       # beta = 0.2 <= 0.2: index
    assert not sel.use_index(201, 1000, 200)   # beta above theta: scan
    assert sel.use_index(0, 10, 0)
    assert not sel.use_index(1, 10, 0)
    assert sel.use_index(10, 10, 1000)


@pytest.mark.parametrize("pct", [1, 2, 5, 10, 20])
def test_recent_window_start_leaves_the_share(pct):
    rng = np.random.default_rng(pct)
    t = rng.integers(0, 1 << 30, 100_000)
    T = sel.recent_start(t, pct)
    share = (t >= T).mean() * 100
    assert abs(share - pct) < 0.01 + 100 / t.size


def test_accuracy_measure_on_a_workload_graph():
    """The Sec. 6.5 measure is a fraction in [0, 1] over the indexed vertices, and it is 1
    when the estimate is exact (every edge at a bucket centre)."""
    el = synth.rmat(synth.scaled(synth.WORKLOADS[2].graph, 14, 1 << 19))
    judged, agree = sel.accuracy(el, 256, 5)
    assert judged > 10 and 0 <= agree <= judged

    class E:
        pass

    c = E()
    c.n = 2
    rng = np.random.default_rng(0x5E5)
    c.t = np.concatenate([[0, 99], rng.integers(0, 100, 500)]).astype(np.uint32)  # unit buckets
    c.src = np.zeros(c.t.size, np.int32)
    c.dst = np.ones(c.t.size, np.int32)
    c.lam = np.ones(c.t.size, np.uint32)
    for pct in (1, 5, 20, 60):
        judged, agree = sel.accuracy(c, 10, pct)
        assert judged == 1 and agree == 1
